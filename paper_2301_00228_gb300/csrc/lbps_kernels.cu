// CUDA kernels of the plane-strain lattice Boltzmann time loop
// (arXiv:2301.00228, algorithm summary of Fig. 3), sm_103a.
//
// One time step is three launches on one stream:
//   boundary newmark  acceleration of each boundary point (Eq. acc_neumann,
//                     from the stresses kept with the state copy, or Eq.
//                     acc_dirichlet) and u, du/dt at t + dt (Eq.
//                     integration);
//   bulk              every interior point: acceleration (Eq. navier),
//                     Newmark, and the pull form of the LBE (Eq. LBE).
//                     Memory-bound stencil: reads copy A once, writes copy B
//                     once;
//   boundary reset    phi, psi at boundary points from differences of the new
//                     u (Eq. psi_phi_at_bound), their populations by Eq.
//                     correction-f, the value each streams into its
//                     interior neighbour (Eq. LBE_mod), and the stresses of
//                     the new u (Eq. strain, Eq. hooke) for the next step.
// Copies A (time t) and B (time t + dt) swap after each step.  Every kernel is
// a template over the population storage policy (lbps_device.cuh): FP32 or
// FP64 planes, or FP32 moments (f^0, J) with the non-equilibrium pair sums in
// 16 bits.
#include <algorithm>
#include <type_traits>

#include "lbps_launch.h"
#ifdef LBPS_CHECKED
#include <utility>
#include <vector>
#endif

namespace lbps {

namespace {

enum {
    FLD_UX = 0, FLD_UY = 1, FLD_VX = 2, FLD_VY = 3, FLD_PHI = 4, FLD_PSI = 5,
    FLD_FPHI = 6, FLD_FPSI = 7, FLD_CONS = 8, FLD_KIN = 9, FLD_STRAIN = 10
};

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return LBPS_LDG(p); }

// ------------------------------------------------------------------ init

// Fig. 3 initialisation: phi = div u, psi = curl u by finite differences of
// u(x, 0) (already copied into copy A), populations at equilibrium (Eq. feq).
template <typename P>
__global__ void init_kernel(Geo g, Consts c, KCof<P> k, View<P> A) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    size_t p = (size_t)j * g.px + i;
    if (!body_at(g, i, j)) {  // void points hold no state: all zero
        for (int q = 0; q < 4; ++q) LBPS_ST(&A.u[(size_t)q * g.plane + p], 0.0);
        const double z[2] = {0.0, 0.0};
        P::store_eq_point(A.f, g.plane, p, c, z, z, z, k);
        return;
    }
    double phi = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
    double psi = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
    double vx = LBPS_LD(&A.u[2 * g.plane + p]), vy = LBPS_LD(&A.u[3 * g.plane + p]);
    // First moments from du/dt (J_phi = -v, J_psi = (-v_y, v_x)), in lattice
    // units Jbar = J dt / dh (c cancels: c^alpha . J / (2 c^2) = e_alpha . Jbar / 2).
    double q = c.dt / c.dh;
    const double sv[2] = {phi, psi}, jx[2] = {-vx * q, -vy * q}, jy[2] = {-vy * q, vx * q};
    P::store_eq_point(A.f, g.plane, p, c, sv, jx, jy, k);
}

// Sets *bad if any of the first `planes` FP64 planes of u holds a
// non-finite value at a lattice point (the input check of the host
// initialisation; the pitch padding is not looked at).
__global__ void finite_check_kernel(Geo g, const double* __restrict__ u, int planes, unsigned* bad) {
    const size_t n = (size_t)g.nx * (size_t)g.ny;
    const size_t total = n * (size_t)planes;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const size_t q = t / n, r = t - q * n;
        const size_t j = r / (size_t)g.nx, i = r - j * (size_t)g.nx;
        if (!isfinite(LBPS_LDG(&u[q * g.plane + j * (size_t)g.px + i]))) atomicOr(bad, 1u);
    }
}

// Size of the lattice first moment J that the initial state implies, for the
// choice of the 16-bit storage scale (the stored non-equilibrium sums are
// smaller): per
// point sqrt(2 a_phi) max(|phi|, |psi|) + (|v_x| + |v_y|) dt / dh (a plane
// wave has |Jbar| = sqrt(2 a_phi) |phi| for the dilatation; the shear part is
// smaller by c_s / c_d).  Maximum over the lattice into *out (FP32 bits of a
// non-negative value, which order like unsigned integers).
__global__ void scale_probe_kernel(Geo g, Consts c, const double* __restrict__ u, double sq, unsigned* out) {
    __shared__ float sh[256];
    int t = threadIdx.y * blockDim.x + threadIdx.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    float est = 0.0f;
    if (i < g.nx && j < g.ny && body_at(g, i, j)) {
        const double* ux = u;
        const double* uy = u + g.plane;
        size_t p = (size_t)j * g.px + i;
        double phi = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
        double psi = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
        double v = fabs(LBPS_LD(&u[2 * g.plane + p])) + fabs(LBPS_LD(&u[3 * g.plane + p]));
        double e = sq * fmax(fabs(phi), fabs(psi)) + v * c.dt / c.dh;
        est = isfinite(e) ? (float)e : 3.0e38f;
    }
    sh[t] = est;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) sh[t] = fmaxf(sh[t], sh[t + w]);
        __syncthreads();
    }
    if (t == 0) atomicMax(out, __float_as_uint(sh[0]));
}

// ------------------------------------------------------------- boundary

// Cauchy stress (Eq. hooke with the strain of Eq. strain) from the four
// differences of u at a point: exx = du_x/dx, eyy = du_y/dy, uxy = du_x/dy,
// uyx = du_y/dx; s = {xx, yy, xy}.
__device__ inline void stress_of(const Consts& c, double exx, double eyy, double uxy, double uyx, double s[3]) {
    double exy = 0.5 * (uxy + uyx);
    double tr = exx + eyy;
    s[0] = c.lam * tr + 2.0 * c.mu * exx;
    s[1] = c.lam * tr + 2.0 * c.mu * eyy;
    s[2] = 2.0 * c.mu * exy;
}

// The same from differences of u at (i, j).
__device__ inline void stress_at(const Geo& g, const Consts& c, const double* ux, const double* uy, int i,
                                 int j, double s[3]) {
    stress_of(c, ddx(ux, g.px, i, j, g, c.inv2h), ddy(uy, g.px, i, j, g, c.inv2h), ddy(ux, g.px, i, j, g, c.inv2h),
              ddx(uy, g.px, i, j, g, c.inv2h), s);
}

// Eq. acc_neumann for the boundary cell of (i, j): the square of side dh
// clipped to the rectangle; one face per existing neighbour r with normal
// pointing to r, length l_kr, stress (sigma_k + sigma_r)/2; external force
// F = int t* da supplied per point.  The stresses come from the stress pass:
// slot b at boundary point b, slot nb + b at its interior neighbour.
// General geometry (reading R14): the cell's side lengths and 1/(rho V_C)
// come with the point; sigma at b is in slot 5b and at its body neighbour in
// direction d in slot 5b + 1 + d; a side facing no
// body neighbour but lying partly in the body carries sigma_k.
__device__ inline void accel_neumann(const Geo& g, const Consts& c, const BNode* __restrict__ bn,
                                     const double* __restrict__ sig, int nb, int b, int i, int j, double fx,
                                     double fy, double& ax, double& ay) {
    const int DX[4] = {1, 0, -1, 0};
    const int DY[4] = {0, 1, 0, -1};
    if (g.general) {
        const int nbm = LBPS_LD(&bn[b].nbmask);
        double sk[3];
        for (int q = 0; q < 3; ++q) sk[q] = LBPS_LD(&sig[(size_t)b * 15 + q]);
        for (int d = 0; d < 4; ++d) {
            const double len = LBPS_LD(&bn[b].l[d]);
            const bool has = (nbm >> d) & 1;
            if (!has && !(len > 0.0)) continue;
            double sr[3];
            for (int q = 0; q < 3; ++q) sr[q] = has ? LBPS_LD(&sig[(size_t)b * 15 + 3 * (1 + d) + q]) : sk[q];
            double sxx = 0.5 * (sk[0] + sr[0]);
            double syy = 0.5 * (sk[1] + sr[1]);
            double sxy = 0.5 * (sk[2] + sr[2]);
            fx += (sxx * DX[d] + sxy * DY[d]) * len;
            fy += (sxy * DX[d] + syy * DY[d]) * len;
        }
        const double inv_m = LBPS_LD(&bn[b].inv_m);
        ax = fx * inv_m;
        ay = fy * inv_m;
        return;
    }
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
// of the stored (a5, copy A) and reset (b5, copy B) populations of the
// source; the equilibrium is taken from f-hat (mode 0) or from f(x_k, t)
// (mode 1).  ALPHA is the direction of travel (1..4), OPP its reverse.
template <int ALPHA, int OPP, typename V>
__device__ inline V stream_from_boundary(const V (&a5)[5], const V (&b5)[5], const KC<V>& k, int set, int mode) {
    V h5[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) h5[q] = mul_rn((V)0.5, add_rn(a5[q], b5[q]));
    if (mode == 0) {
        V sh = sum5(h5[0], h5[1], h5[2], h5[3], h5[4]);
        return fma_rn(k.two_a[set], sh, -h5[OPP]);  // 2 f_eq(f-hat) - f-hat = 2 a s-hat - f-hat^opp
    }
    V sa = sum5(a5[0], a5[1], a5[2], a5[3], a5[4]);
    V ej = sub_rn(a5[ALPHA], a5[OPP]);              // e_alpha . Jbar(x_k, t)
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

// The boundary work of a step runs in two passes over the perimeter list,
// each one thread per boundary point b at (i, j):
//   newmark  acceleration of b (Eq. acc_neumann, from the stresses of copy A,
//            or Eq. acc_dirichlet) and u(t + dt) at b;
//   (the interior kernel runs here: u(t + dt) at every interior point)
//   reset    phi, psi from differences of u(t + dt) (Eq. psi_phi_at_bound),
//            populations by Eq. correction-f, the value b streams into its
//            interior neighbour (Eq. LBE_mod), written over the population the
//            interior kernel put there, and the stresses of u(t + dt) that
//            the next step's Eq. acc_neumann reads, into copy B.
// Each copy thus carries the stresses of its own u; the stress pass below
// computes them where u was set otherwise (initialisation).

// sigma at b (slot b of a rectangle, 5b of a general geometry).
__device__ inline void store_point_stress(const Geo& g, double* __restrict__ sig, int b, const double s[3]) {
    const size_t o = (size_t)b * (g.general ? 15 : 3);
    for (int q = 0; q < 3; ++q) LBPS_ST(&sig[o + q], s[q]);
}

// sigma at the neighbours of b that its Eq. acc_neumann reads besides the
// boundary points: the interior neighbour of a rectangle's edge point (slot
// nb + b), the body neighbours of a general boundary point (slot 5b + 1 + d).
__device__ inline void neighbour_stresses(const Geo& g, const Consts& c, const double* ux, const double* uy,
                                          const BNode* __restrict__ bn, int nb, double* __restrict__ sig, int b,
                                          int i, int j) {
    double s[3];
    if (g.general) {
        const int DX[4] = {1, 0, -1, 0};
        const int DY[4] = {0, 1, 0, -1};
        const int nbm = LBPS_LD(&bn[b].nbmask);
        for (int d = 0; d < 4; ++d) {
            if (!((nbm >> d) & 1)) continue;
            stress_at(g, c, ux, uy, wrap(i + DX[d], g.nx), wrap(j + DY[d], g.ny), s);
            for (int q = 0; q < 3; ++q) LBPS_ST(&sig[(size_t)b * 15 + 3 * (1 + d) + q], s[q]);
        }
        return;
    }
    const int dir = inward_dir(i, j, g);
    if (dir != 0) {
        const int DX[5] = {0, 1, 0, -1, 0};
        const int DY[5] = {0, 0, 1, 0, -1};
        stress_at(g, c, ux, uy, i + DX[dir], j + DY[dir], s);
        for (int q = 0; q < 3; ++q) LBPS_ST(&sig[((size_t)nb + b) * 3 + q], s[q]);
    }
}

__device__ inline void boundary_stress(const Geo& g, const Consts& c, const double* ux, const double* uy,
                                       const BNode* __restrict__ bn, int nb, double* __restrict__ sig, int b) {
    const int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    double s[3];
    stress_at(g, c, ux, uy, i, j, s);
    store_point_stress(g, sig, b, s);
    neighbour_stresses(g, c, ux, uy, bn, nb, sig, b, i, j);
}

// tstep: the lattice's step counter n (device memory); time-dependent data
// take the Neumann force at t_n and the Dirichlet target at t_{n+1}.
template <typename P>
__device__ inline void boundary_newmark(const Geo& g, const Consts& c, const View<P>& A, const View<P>& B,
                                        const BNode* __restrict__ bn, int nb,
                                        const double* __restrict__ sig,
                                        const unsigned long long* __restrict__ tstep, int b) {
    int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    const int btype = LBPS_LD(&bn[b].type);
    const double n = (double)LBPS_LD(tstep);
    const double sc = btype == DIRICHLET ? load_factor(c, 1, (n + 1.0) * c.dt) : load_factor(c, 0, n * c.dt);
    const double bx = sc * LBPS_LD(&bn[b].bx), by = sc * LBPS_LD(&bn[b].by);
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
        accel_neumann(g, c, bn, sig, nb, b, i, j, bx, by, ax, ay);
    }
    double ux1, uy1, vx1, vy1;
    newmark(LBPS_LD(&ux[p]), LBPS_LD(&vx[p]), ax, c, ux1, vx1);
    newmark(LBPS_LD(&uy[p]), LBPS_LD(&vy[p]), ay, c, uy1, vy1);
    LBPS_ST(&B.u[p], ux1);
    LBPS_ST(&B.u[g.plane + p], uy1);
    LBPS_ST(&B.u[2 * g.plane + p], vx1);
    LBPS_ST(&B.u[3 * g.plane + p], vy1);
}

// bc_j_mode 1: J(x_k, t) of Eq. correction-f is the first moment of the
// populations the plain LBE (Eq. LBE, from copy A) streams into (i, j):
// direction alpha arrives from the body neighbour at x - e_alpha as
// 2 a s - f^opp there (tau = dt/2); a direction whose source is outside the
// body keeps the point's own stored population (own5).
template <typename P>
__device__ inline void partial_stream_moment(const Geo& g, const KCof<P>& k, const View<P>& A, int i, int j,
                                             const typename P::V (&own5)[2][5], double (&jx)[2],
                                             double (&jy)[2]) {
    using V = typename P::V;
    const int SX[5] = {0, -1, 0, 1, 0};  // source offset x - e_alpha
    const int SY[5] = {0, 0, -1, 0, 1};
    const int OPP[5] = {0, 3, 4, 1, 2};
    V in5[2][5];
#pragma unroll
    for (int set = 0; set < 2; ++set)
#pragma unroll
        for (int q = 1; q < 5; ++q) in5[set][q] = own5[set][q];
    for (int q = 1; q < 5; ++q) {
        const int si = i + SX[q], sj = j + SY[q];
        if (!body_at(g, si, sj)) continue;
        typename P::Raw r;
        P::load_raw(A.f, g.plane, (size_t)wrap(sj, g.ny) * g.px + wrap(si, g.nx), true, r);
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            V f5[5];
            P::decode(r, set, k, f5);
            in5[set][q] = fma_rn(k.two_a[set], sum5(f5[0], f5[1], f5[2], f5[3], f5[4]), -f5[OPP[q]]);
        }
    }
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        jx[set] = (double)in5[set][1] - (double)in5[set][3];
        jy[set] = (double)in5[set][2] - (double)in5[set][4];
    }
}

// The populations boundary point (i, j) streams into its interior
// neighbours, the directions d (0: +x, 1: +y, 2: -x, 3: -y) set in mask, from
// its populations at t (a5s) and after the reset (b5s) (Eq. LBE_mod).
template <typename P>
__device__ inline void stream_out(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& B, int i, int j,
                                  int mask, const typename P::V (&a5s)[2][5], const typename P::V (&b5s)[2][5]) {
    using V = typename P::V;
    const int DXS[4] = {1, 0, -1, 0};
    const int DYS[4] = {0, 1, 0, -1};
    for (int d = 0; d < 4; ++d) {
        if (!((mask >> d) & 1)) continue;
        V v[2];
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            switch (d) {
            case 0: v[set] = stream_from_boundary<1, 3>(a5s[set], b5s[set], k, set, c.bc_feq_mode); break;
            case 1: v[set] = stream_from_boundary<2, 4>(a5s[set], b5s[set], k, set, c.bc_feq_mode); break;
            case 2: v[set] = stream_from_boundary<3, 1>(a5s[set], b5s[set], k, set, c.bc_feq_mode); break;
            default: v[set] = stream_from_boundary<4, 2>(a5s[set], b5s[set], k, set, c.bc_feq_mode); break;
            }
        }
        const size_t pin = (size_t)wrap(j + DYS[d], g.ny) * g.px + wrap(i + DXS[d], g.nx);
        P::store1_both(B.f, g.plane, pin, d + 1, v, k);
    }
}

template <typename P>
__device__ inline bool boundary_reset(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& A,
                                      const View<P>& B, const BNode* __restrict__ bn, int nb, int b) {
    using V = typename P::V;
    int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    size_t p = (size_t)j * g.px + i;
    const double* ux1 = B.u;
    const double* uy1 = B.u + g.plane;
    // The populations at t (copy A's boundary mirror, entry b, coalesced
    // along the boundary list) and the streaming mask, loaded first: nothing
    // below writes them, and issued here their latency overlaps the
    // differences and the stress stores instead of following them.
    const int smask = LBPS_LD(&bn[b].smask);
    typename P::Raw ra, rb;
    P::load_raw(A.m, g.mplane, (size_t)b, true, ra);
    // Eq. psi_phi_at_bound: differences of u(t + dt) at (i, j).
    Sten sx = stencil_x(g, i, j), sy = stencil_y(g, i, j);
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
    const double exx = mul_rn(dux_dx, c.inv2h), eyy = mul_rn(duy_dy, c.inv2h);
    const double uxy = mul_rn(dux_dy, c.inv2h), uyx = mul_rn(duy_dx, c.inv2h);
    const double phi = exx + eyy;
    const double psi = uyx - uxy;
    // sigma of u(t + dt) at b (from the same differences) and at the
    // neighbours Eq. acc_neumann reads, into copy B for the next step
    {
        double s[3];
        stress_of(c, exx, eyy, uxy, uyx, s);
        store_point_stress(g, B.s, b, s);
        neighbour_stresses(g, c, ux1, uy1, bn, nb, B.s, b, i, j);
    }
    // Eq. correction-f with J(x_k, t) of the stored populations, then the value
    // this point streams into each interior neighbour (Eq. LBE_mod): the
    // population travelling that way, replacing what the interior kernel
    // wrote there (a rectangle's edge point has one such neighbour, a corner
    // none; next to a hole a point may have several).
    // The reset populations go to the lattice and to copy B's mirror.
    V a5s[2][5], b5s[2][5];
    const double sv[2] = {phi, psi};
    double jx[2], jy[2];
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        P::decode(ra, set, k, a5s[set]);
        jx[set] = (double)a5s[set][1] - (double)a5s[set][3];
        jy[set] = (double)a5s[set][2] - (double)a5s[set][4];
    }
    if (c.bc_j_mode == 1) partial_stream_moment<P>(g, k, A, i, j, a5s, jx, jy);
    P::eq_raw(p, c, sv, jx, jy, k, rb);
    P::store_raw(B.f, g.plane, p, rb);
    P::store_raw(B.m, g.mplane, (size_t)b, rb);
    if (smask)
#pragma unroll
        for (int set = 0; set < 2; ++set) P::decode(rb, set, k, b5s[set]);
    // a policy whose words hold both pairs of a point leaves the y streams to
    // a second pass (boundary_stream_y): two boundary points may stream into
    // one point along x and along y
    stream_out<P>(g, c, k, B, i, j, P::kSplitStream ? (smask & 5) : smask, a5s, b5s);
    return !isfinite((V)phi + (V)psi);
}

// The y streams of the reset for PopBfp13 (P::kSplitStream), in a pass after
// the one that wrote everything else: the values depend only on the boundary
// point's populations at t (copy A's mirror) and those the reset stored for
// t + dt (copy B's mirror), which that pass left as they are.
template <typename P>
__device__ inline void boundary_stream_y(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& A,
                                         const View<P>& B, const BNode* __restrict__ bn, int b) {
    using V = typename P::V;
    const int smask = LBPS_LD(&bn[b].smask) & 10;
    if (!smask) return;
    const int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    typename P::Raw ra, rb;
    P::load_raw(A.m, g.mplane, (size_t)b, true, ra);
    P::load_raw(B.m, g.mplane, (size_t)b, true, rb);
    V a5s[2][5], b5s[2][5];
#pragma unroll
    for (int set = 0; set < 2; ++set) {
        P::decode(ra, set, k, a5s[set]);
        P::decode(rb, set, k, b5s[set]);
    }
    stream_out<P>(g, c, k, B, i, j, smask, a5s, b5s);
}

template <typename P>
__global__ void __launch_bounds__(128) boundary_stress_kernel(Geo g, Consts c, View<P> A,
                                                              const BNode* __restrict__ bn, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) boundary_stress(g, c, A.u, A.u + g.plane, bn, nb, A.s, b);
}

template <typename P>
__global__ void __launch_bounds__(128) boundary_newmark_kernel(Geo g, Consts c, View<P> A, View<P> B,
                                                               const BNode* __restrict__ bn, int nb,
                                                               const unsigned long long* __restrict__ tstep) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) boundary_newmark(g, c, A, B, bn, nb, A.s, tstep, b);
}

// The last pass of a step also advances the step counter (one thread; no
// other thread of the pass reads it).
template <typename P>
__global__ void __launch_bounds__(128) boundary_reset_kernel(Geo g, Consts c, KCof<P> k, View<P> A, View<P> B,
                                                             const BNode* __restrict__ bn, int nb, unsigned* flag,
                                                             unsigned long long* tstep) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb && boundary_reset(g, c, k, A, B, bn, nb, b)) atomicOr(flag, 1u);
    if (b == 0) LBPS_ST(tstep, LBPS_LD(tstep) + 1ull);
}

template <typename P>
__global__ void __launch_bounds__(128) boundary_stream_y_kernel(Geo g, Consts c, KCof<P> k, View<P> A, View<P> B,
                                                                const BNode* __restrict__ bn, int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) boundary_stream_y(g, c, k, A, B, bn, b);
}

// Copies the populations of every boundary point of copy A into A's boundary
// mirror.  Run after the kernels that write them in place (initialisation,
// synchronisation); the reset pass keeps the mirror current otherwise.
template <typename P>
__global__ void __launch_bounds__(128) boundary_mirror_kernel(Geo g, View<P> A, const BNode* __restrict__ bn,
                                                              int nb) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int i = LBPS_LD(&bn[b].i), j = LBPS_LD(&bn[b].j);
    typename P::Raw r;
    P::load_raw(A.f, g.plane, (size_t)j * g.px + i, true, r);
    P::store_raw(A.m, g.mplane, (size_t)b, r);
}

// ---------------------------------------------------------------- bulk

// Bulk kernel: each warp owns a strip of kStripCols output columns and marches
// along y over kRowsPerWarp rows.  Lane l holds column xs - 1 + l, so lanes 0
// and 31 are halo lanes whose values reach their neighbours by shuffles; the
// rows above and below stay in registers, and the populations are prefetched
// two rows ahead (in their stored form, decoded when the row window shifts).
// Every lattice point's words are read once per launch (plus the two halo
// columns and two halo rows of each strip).
constexpr int kStripCols = 30;
static_assert(kStripCols == kBatchStripCols, "one strip width for the single-lattice and batched kernels");
constexpr int kWarpsPerBlock = 4;

template <typename P>
__device__ __forceinline__ void decode_row(const typename P::Raw& r, const KCof<P>& k,
                                           typename P::V (&f)[2][5]) {
#pragma unroll
    for (int s = 0; s < 2; ++s) P::decode(r, s, k, f[s]);
}

__device__ __forceinline__ void load_uv(const double* __restrict__ U, size_t plane, size_t p, bool ok,
                                        double (&u)[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = ok ? ld(U + (size_t)q * plane + p) : 0.0;
}

// An output window of the interior kernel: columns [x0, x1), rows [y0, y1).
struct Win {
    int x0, x1, y0, y1;
};

// The moving populations of interior point (i, j) (plane offset p) that
// stream in from boundary points and that the reset pass overwrites: 1 f^1
// (from i - 1), 2 f^3 (from i + 1), 4 f^2 (from j - 1), 8 f^4 (from j + 1).
// A rectangle's boundary points are its non-periodic edges; a general
// geometry marks them in its node-type plane.
__device__ __forceinline__ int streamed_in(const Geo& g, int i, int j, size_t p) {
    if (!g.general) {
        int m = 0;
        if (!g.periodic_x) m |= (i == 1 ? 1 : 0) | (i == g.nx - 2 ? 2 : 0);
        if (!g.periodic_y) m |= (j == 1 ? 4 : 0) | (j == g.ny - 2 ? 8 : 0);
        return m;
    }
    auto bnd = [&](size_t q) {
        const int t = LBPS_LDG(&g.type[q]);
        return t == NEUMANN || t == DIRICHLET;
    };
    const size_t row = p - (size_t)i;
    return (bnd(row + (size_t)wrap(i - 1, g.nx)) ? 1 : 0) | (bnd(row + (size_t)wrap(i + 1, g.nx)) ? 2 : 0) |
           (bnd((size_t)wrap(j - 1, g.ny) * g.px + (size_t)i) ? 4 : 0) |
           (bnd((size_t)wrap(j + 1, g.ny) * g.px + (size_t)i) ? 8 : 0);
}

// One warp's strip: output columns [xs, xs + kStripCols) of rows [j0, j1).
// Returns true in lanes that produced a non-finite value.  All 32 lanes of
// the warp must call it together (warp shuffles).  UVD: how many rows ahead u
// and du/dt are prefetched (1 or 2; the populations always 2).  WIN: writes
// only points inside the window w (the frame passes of a two-step sweep).
template <typename P, int UVD, bool WIN = false>
__device__ __forceinline__ bool bulk_strip(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& A,
                                           const View<P>& B, int xs, int j0, int j1, Win w = Win{0, 0, 0, 0}) {
    using V = typename P::V;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int xl = xs - 1 + lane;
    const bool col_ok = g.periodic_x ? (xl <= g.nx) : (xl >= 0 && xl < g.nx);
    const int col = col_ok ? wrap(xl, g.nx) : 0;
    const bool out_lane = lane >= 1 && lane <= kStripCols && xl < g.nx &&
                          (g.periodic_x || (xl > 0 && xl < g.nx - 1)) && (!WIN || (xl >= w.x0 && xl < w.x1));
    const size_t PL = g.plane;

    auto row_ok = [&](int j) { return g.periodic_y || (j >= 0 && j < g.ny); };
    auto row_of = [&](int j) { return g.periodic_y ? wrap(j, g.ny) : j; };
    // Offsets are formed only for rows inside the lattice (rows outside are
    // clamped; their loads are masked), so no address ever leaves the planes
    // even where a masked load is issued unconditionally.
    auto at = [&](int j) { return (size_t)min(max(row_of(j), 0), g.ny - 1) * (size_t)g.px + (size_t)col; };

    V Ps[2], Pf4[2];                          // row j - 1: moment and f^4
    V Cf[2][5], Cs[2], Cm[2];                 // row j
    V Nf[2][5];                               // row j + 1
    typename P::Raw Qr;                       // row j + 2 (in flight, stored form)
    double Cu[4], Nu[4], Qu[4];               // u, du/dt of rows j, j + 1, j + 2
    {
        V t[2][5];
        P::load_raw(A.f, PL, at(j0 - 1), col_ok && row_ok(j0 - 1), Qr);
        decode_row<P>(Qr, k, t);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Ps[s] = sum5(t[s][0], t[s][1], t[s][2], t[s][3], t[s][4]);
            Pf4[s] = t[s][4];
        }
    }
    P::load_raw(A.f, PL, at(j0), col_ok, Qr);
    decode_row<P>(Qr, k, Cf);
    P::load_raw(A.f, PL, at(j0 + 1), col_ok && row_ok(j0 + 1), Qr);
    decode_row<P>(Qr, k, Nf);
    load_uv(A.u, PL, at(j0), out_lane, Cu);
    if (UVD == 2) load_uv(A.u, PL, at(j0 + 1), out_lane && j0 + 1 < j1, Nu);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        Cm[s] = add_rn(add_rn(Cf[s][1], Cf[s][2]), add_rn(Cf[s][3], Cf[s][4]));
        Cs[s] = add_rn(Cf[s][0], Cm[s]);
    }
    bool bad = false;
    for (int j = j0; j < j1; ++j) {
        // prefetch: populations two rows ahead, u and du/dt one row ahead
        P::load_raw(A.f, PL, at(j + 2), col_ok && row_ok(j + 2) && j + 2 <= j1, Qr);
        if (UVD == 2)
            load_uv(A.u, PL, at(j + 2), out_lane && j + 2 < j1, Qu);
        else
            load_uv(A.u, PL, at(j + 1), out_lane && j + 1 < j1, Nu);
        V Nm[2], Ns[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            Nm[s] = add_rn(add_rn(Nf[s][1], Nf[s][2]), add_rn(Nf[s][3], Nf[s][4]));
            Ns[s] = add_rn(Nf[s][0], Nm[s]);
        }
        const bool row_interior = (g.periodic_y || (j > 0 && j < g.ny - 1)) && (!WIN || (j >= w.y0 && j < w.y1));
        if (row_interior) {  // warp-uniform
            V sW[2], sE[2], out[2][5];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sW[s] = __shfl_up_sync(FULL, Cs[s], 1);
                sE[s] = __shfl_down_sync(FULL, Cs[s], 1);
                V f3W = __shfl_up_sync(FULL, Cf[s][3], 1);
                V f1E = __shfl_down_sync(FULL, Cf[s][1], 1);
                // rest population: 2 a0 s - f0 = f0 + (2 a0 m - 8 a f0)
                out[s][0] = add_rn(Cf[s][0], fma_rn(k.two_a0[s], Cm[s], -mul_rn(k.eight_a[s], Cf[s][0])));
                // moving populations: f^alpha(x) = 2 a s(x - e_alpha) - f^opp(x - e_alpha)
                // (for sources on the boundary the reset pass overwrites them)
                out[s][1] = fma_rn(k.two_a[s], sW[s], -f3W);
                out[s][3] = fma_rn(k.two_a[s], sE[s], -f1E);
                out[s][2] = fma_rn(k.two_a[s], Ps[s], -Pf4[s]);
                out[s][4] = fma_rn(k.two_a[s], Ns[s], -Nf[s][2]);
            }
            const size_t p = at(j);
            // general geometry: only interior points (boundary and void points
            // are the boundary passes' or stay zero)
            if (out_lane && (!g.general || LBPS_LDG(&g.type[p]) == 0)) {
                double ax, ay;
                accel_interior<V>(sW[0], sE[0], Ps[0], Ns[0], sW[1], sE[1], Ps[1], Ns[1], k, ax, ay);
                double u1[4];
                newmark(Cu[0], Cu[2], ax, c, u1[0], u1[2]);
                newmark(Cu[1], Cu[3], ay, c, u1[1], u1[3]);
                if constexpr (P::kSplitStream)
                    P::store_point_pins(B.f, PL, p, out, k, streamed_in(g, col, j, p));
                else
                    P::store_point(B.f, PL, p, out, k);
#pragma unroll
                for (int q = 0; q < 4; ++q) LBPS_ST(&B.u[(size_t)q * PL + p], u1[q]);
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
            for (int q = 0; q < 5; ++q) Cf[s][q] = Nf[s][q];
        }
        decode_row<P>(Qr, k, Nf);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Cu[q] = Nu[q];
            if (UVD == 2) Nu[q] = Qu[q];
        }
    }
    return bad;
}

template <typename P, int MINB, int UVD>
__global__ void __launch_bounds__(128, MINB) bulk_kernel(Geo g, Consts c, KCof<P> k, View<P> A, View<P> B,
                                                         unsigned* flag, int rows_per_warp) {
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int xs = warp * kStripCols;
    if (xs >= g.nx) return;  // whole warp
    const int j0 = blockIdx.y * rows_per_warp;
    const int j1 = min(j0 + rows_per_warp, g.ny);
    // General geometry: a warp whose rows all lie in its strip's run of rows
    // without interior points (inside a hole) has nothing to write, and no
    // interior point reads those rows: it returns before loading them.
    if (g.gap && j0 >= LBPS_LD(&g.gap[2 * warp]) && j1 <= LBPS_LD(&g.gap[2 * warp + 1])) return;
    const bool bad = bulk_strip<P, UVD>(g, c, k, A, B, xs, j0, j1);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// ------------------------------------------------- two steps per sweep

// The interior kernel restricted to the window w: strips s0 .. s0 + nstrips - 1,
// rows [jb, je) in chunks of `rows` (the frame passes of a two-step sweep).
template <typename P, int MINB, int UVD>
__global__ void __launch_bounds__(128, MINB) frame_kernel(Geo g, Consts c, KCof<P> k, View<P> A, View<P> B,
                                                          unsigned* flag, int s0, int nstrips, int jb, int je,
                                                          int rows, Win w) {
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (warp >= nstrips) return;  // whole warp
    const int xs = (s0 + warp) * kStripCols;
    const int j0 = jb + blockIdx.y * rows;
    const int j1 = min(j0 + rows, je);
    if (j0 >= j1) return;
    const bool bad = bulk_strip<P, UVD, true>(g, c, k, A, B, xs, j0, j1, w);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

constexpr int kPairCols = 28;  // output columns of a warp in the two-step kernel
constexpr int kDeep = 3;       // the two-step kernel writes points at least this far from every edge

// Two time steps of the deep interior of a rectangle (no periodic axis, no
// void points) in one sweep: the warp marches its strip's rows computing step
// n + 1 from copy A (state n) exactly as bulk_strip does, rounds it to its
// stored form as a store and reload would, and from those values step n + 2,
// which it writes to copy B.  Lanes are columns xs - 2 .. xs + 29: step n + 1
// is valid in lanes 1..30, step n + 2 in lanes 2..29 (output columns xs ..
// xs + 27).  Rows [j0, j1) need step n + 1 at rows j0 - 1 .. j1 and state n
// at rows j0 - 2 .. j1 + 1.  A point at least kDeep from every edge depends
// at step n + 2 only on interior points at step n + 1 that are at least 2
// from the edges, which the boundary reset of step n does not touch, so
// nothing here needs the boundary passes.
template <typename P>
__device__ __forceinline__ bool pair_strip(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& A,
                                           const View<P>& B, int xs, int j0, int j1) {
    using V = typename P::V;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int xl = xs - 2 + lane;
    const bool col_ok = xl < g.nx;             // xl >= 1 always (xs >= kDeep)
    const int col = col_ok ? xl : g.nx - 1;
    const bool out_lane = lane >= 2 && lane < 2 + kPairCols && xl < g.nx - kDeep;
    const size_t PL = g.plane;
    auto at = [&](int j) { return (size_t)j * (size_t)g.px + (size_t)col; };

    // step n (state n, read): rows r - 1, r, r + 1 and r + 2 in flight
    V P0s[2], P0f4[2];
    V C0f[2][5], C0s[2], C0m[2];
    V N0f[2][5];
    typename P::Raw Qr;
    // step n + 1: rows r - 2 (moment, f^4), r - 1 (all); filled by the first
    // two iterations, which write nothing
    V P1s[2] = {}, P1f4[2] = {};
    V C1f[2][5] = {}, C1s[2] = {}, C1m[2] = {};
    double C1u[4] = {};   // u, du/dt of row r - 1 at step n (loaded one iteration ahead)
    V C1a[2] = {};        // the accelerations of row r - 1 at step n

    {
        V t[2][5];
        P::load_raw(A.f, PL, at(j0 - 2), col_ok, Qr);
        decode_row<P>(Qr, k, t);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            P0s[s] = sum5(t[s][0], t[s][1], t[s][2], t[s][3], t[s][4]);
            P0f4[s] = t[s][4];
        }
    }
    P::load_raw(A.f, PL, at(j0 - 1), col_ok, Qr);
    decode_row<P>(Qr, k, C0f);
    P::load_raw(A.f, PL, at(j0), col_ok, Qr);
    decode_row<P>(Qr, k, N0f);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        C0m[s] = add_rn(add_rn(C0f[s][1], C0f[s][2]), add_rn(C0f[s][3], C0f[s][4]));
        C0s[s] = add_rn(C0f[s][0], C0m[s]);
    }
    bool bad = false;
    // r: the row of step n + 1 computed this iteration; step n + 2 at r - 1
    for (int r = j0 - 1; r <= j1; ++r) {
        P::load_raw(A.f, PL, at(r + 2), col_ok && r + 2 <= j1 + 1, Qr);
        // u, du/dt only where a point is written: row r, used by the next
        // iteration's second stage
        double Nu[4];
        load_uv(A.u, PL, at(r), out_lane && r >= j0 && r < j1, Nu);
        V N0m[2], N0s[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            N0m[s] = add_rn(add_rn(N0f[s][1], N0f[s][2]), add_rn(N0f[s][3], N0f[s][4]));
            N0s[s] = add_rn(N0f[s][0], N0m[s]);
        }
        // step n + 1 at row r (bulk_strip's arithmetic)
        V N1f[2][5], N1a[2];
        {
            V sW[2], sE[2], out[2][5];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sW[s] = __shfl_up_sync(FULL, C0s[s], 1);
                sE[s] = __shfl_down_sync(FULL, C0s[s], 1);
                V f3W = __shfl_up_sync(FULL, C0f[s][3], 1);
                V f1E = __shfl_down_sync(FULL, C0f[s][1], 1);
                out[s][0] = add_rn(C0f[s][0], fma_rn(k.two_a0[s], C0m[s], -mul_rn(k.eight_a[s], C0f[s][0])));
                out[s][1] = fma_rn(k.two_a[s], sW[s], -f3W);
                out[s][3] = fma_rn(k.two_a[s], sE[s], -f1E);
                out[s][2] = fma_rn(k.two_a[s], P0s[s], -P0f4[s]);
                out[s][4] = fma_rn(k.two_a[s], N0s[s], -N0f[s][2]);
            }
            // the accelerations at step n, for the second stage, which
            // integrates both steps at once
            accel_interior_v<V>(sW[0], sE[0], P0s[0], N0s[0], sW[1], sE[1], P0s[1], N0s[1], k, N1a[0], N1a[1]);
            // as stored at row r and read back
            typename P::Raw q;
            P::pack(at(r), out, k, q);
            decode_row<P>(q, k, N1f);
        }
        V N1m[2], N1s[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            N1m[s] = add_rn(add_rn(N1f[s][1], N1f[s][2]), add_rn(N1f[s][3], N1f[s][4]));
            N1s[s] = add_rn(N1f[s][0], N1m[s]);
        }
        // step n + 2 at row r - 1
        if (r - 1 >= j0) {  // warp-uniform
            V sW[2], sE[2], out[2][5];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                sW[s] = __shfl_up_sync(FULL, C1s[s], 1);
                sE[s] = __shfl_down_sync(FULL, C1s[s], 1);
                V f3W = __shfl_up_sync(FULL, C1f[s][3], 1);
                V f1E = __shfl_down_sync(FULL, C1f[s][1], 1);
                out[s][0] = add_rn(C1f[s][0], fma_rn(k.two_a0[s], C1m[s], -mul_rn(k.eight_a[s], C1f[s][0])));
                out[s][1] = fma_rn(k.two_a[s], sW[s], -f3W);
                out[s][3] = fma_rn(k.two_a[s], sE[s], -f1E);
                out[s][2] = fma_rn(k.two_a[s], P1s[s], -P1f4[s]);
                out[s][4] = fma_rn(k.two_a[s], N1s[s], -N1f[s][2]);
            }
            if (out_lane) {
                const size_t p = at(r - 1);
                V ax, ay;
                accel_interior_v<V>(sW[0], sE[0], P1s[0], N1s[0], sW[1], sE[1], P1s[1], N1s[1], k, ax, ay);
                double u2[4];
                newmark2(C1u[0], C1u[2], C1a[0], ax, c, u2[0], u2[2]);
                newmark2(C1u[1], C1u[3], C1a[1], ay, c, u2[1], u2[3]);
                P::store_point(B.f, PL, p, out, k);
#pragma unroll
                for (int q = 0; q < 4; ++q) LBPS_ST(&B.u[(size_t)q * PL + p], u2[q]);
                bad |= !isfinite(out[0][0] + out[1][0]);
            }
        }
        // shift both windows
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            P1s[s] = C1s[s];
            P1f4[s] = C1f[s][4];
            C1s[s] = N1s[s];
            C1m[s] = N1m[s];
#pragma unroll
            for (int q = 0; q < 5; ++q) C1f[s][q] = N1f[s][q];
            P0s[s] = C0s[s];
            P0f4[s] = C0f[s][4];
            C0s[s] = N0s[s];
            C0m[s] = N0m[s];
#pragma unroll
            for (int q = 0; q < 5; ++q) C0f[s][q] = N0f[s][q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) C1u[q] = Nu[q];
        C1a[0] = N1a[0];
        C1a[1] = N1a[1];
        decode_row<P>(Qr, k, N0f);
    }
    return bad;
}

template <typename P, int MINB>
__global__ void __launch_bounds__(128, MINB) pair_kernel(Geo g, Consts c, KCof<P> k, View<P> A, View<P> B,
                                                         unsigned* flag, int rows_per_warp) {
    const int warp = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const int xs = kDeep + warp * kPairCols;
    if (xs >= g.nx - kDeep) return;  // whole warp
    const int j0 = kDeep + blockIdx.y * rows_per_warp;
    const int j1 = min(j0 + rows_per_warp, g.ny - kDeep);
    if (j0 >= j1) return;
    const bool bad = pair_strip<P>(g, c, k, A, B, xs, j0, j1);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// --------------------------------------------------------------- batches

// The boundary passes of a step (1 Newmark, 2 reset, 3 the y streams of the
// reset where P::kSplitStream) over the boundary points of every lattice in
// the batch (one thread per point).
template <typename P>
__global__ void __launch_bounds__(128) boundary_batch_kernel(const DomDesc<P>* __restrict__ dd,
                                                             const BndTask* __restrict__ tasks, int ntasks,
                                                             int parity, int pass, int stage) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntasks) return;
    const BndTask tk = tasks[t];
    const DomDesc<P>& d = dd[tk.dom];
    const int a = d.cur ^ parity;
    // the copies the pass reads and writes (stage: see launch_boundary_batch)
    const View<P>& S = stage == 2 ? d.x : d.v[a];
    const View<P>& D = stage == 1 ? d.x : d.v[a ^ 1];
    if (pass == 1)
        boundary_newmark(d.g, d.c, S, D, d.bn, d.nb, S.s, d.tstep, tk.b);
    else if (pass == 3)
        boundary_stream_y(d.g, d.c, d.k, S, D, d.bn, tk.b);
    else {
        if (boundary_reset(d.g, d.c, d.k, S, D, d.bn, d.nb, tk.b)) atomicOr(d.flag, 1u);
        if (tk.b == 0) LBPS_ST(d.tstep, LBPS_LD(d.tstep) + 1ull);
    }
}

// The interior of every lattice in the batch: a persistent grid (as many
// blocks as fit on the GPU at once) whose warps take strip tasks from the
// work list through the counter *next (zero before the launch) until none is
// left, so no wave of short tasks leaves the GPU half idle at the end.  Each
// warp keeps the descriptor of the lattice it works on in shared memory and
// copies a new one only when the next task belongs to another lattice.
template <typename P, int MINB, int UVD>
__global__ void __launch_bounds__(128, MINB) bulk_batch_kernel(const DomDesc<P>* __restrict__ dd,
                                                               const BulkTask* __restrict__ tasks, int ntasks,
                                                               const BndTask* __restrict__ btasks, int parity,
                                                               unsigned* next) {
    __shared__ DomDesc<P> sd[kWarpsPerBlock];
    const unsigned FULL = 0xffffffffu;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cached = -1;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(next, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= (unsigned)ntasks) break;  // whole warp
        const BulkTask tk = tasks[t];
        if (tk.j0 < 0) {
            // Newmark task (warp-uniform): boundary points tk.xs .. tk.xs +
            // tk.j1 - 1 of the boundary work list, one per lane.  It reads
            // copy A and writes only boundary u, du/dt of copy B, which no
            // strip task touches; the reset pass after this kernel reads them.
            if (lane < tk.j1) {
                const BndTask bt = btasks[tk.xs + lane];
                const DomDesc<P>& d = dd[bt.dom];
                const int a = d.cur ^ parity;
                boundary_newmark(d.g, d.c, d.v[a], d.v[a ^ 1], d.bn, d.nb, d.v[a].s, d.tstep, bt.b);
            }
            continue;
        }
        if (tk.dom != cached) {
            __syncwarp();  // every lane is done with the previous descriptor
            const unsigned* src = reinterpret_cast<const unsigned*>(dd + tk.dom);
            unsigned* dst = reinterpret_cast<unsigned*>(sd + wid);
            for (int q = lane; q < (int)(sizeof(DomDesc<P>) / 4); q += 32) dst[q] = src[q];
            __syncwarp();
            cached = tk.dom;
        }
        const DomDesc<P>& d = sd[wid];
        const int a = d.cur ^ parity;
        bool bad = bulk_strip<P, UVD>(d.g, d.c, d.k, d.v[a], d.v[a ^ 1], tk.xs, tk.j0, tk.j1);
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(d.flag, 1u);
    }
}

// Two steps per sweep for every lattice of a batch: one stage of a pair (see
// launch_pair_batch).  The tasks are those of pair_kernel, frame_kernel and
// boundary_newmark_kernel on each lattice, so each lattice gets the same bits
// as run on its own with two steps per sweep.  Frame strips take the shape
// that loads u one row ahead (the results do not depend on it).
template <typename P, int MINB>
__global__ void __launch_bounds__(128, MINB) pair_batch_kernel(const DomDesc<P>* __restrict__ dd,
                                                               const PairTask* __restrict__ tasks, int ntasks,
                                                               const BndTask* __restrict__ btasks, int parity,
                                                               int stage, unsigned* next) {
    __shared__ DomDesc<P> sd[kWarpsPerBlock];
    const unsigned FULL = 0xffffffffu;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int cached = -1;
    for (;;) {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(next, 1u);
        t = __shfl_sync(FULL, t, 0);
        if (t >= (unsigned)ntasks) break;  // whole warp
        const PairTask tk = tasks[t];
        if (tk.kind == kNewmarkTask) {
            if (lane < tk.j1) {
                const BndTask bt = btasks[tk.xs + lane];
                const DomDesc<P>& d = dd[bt.dom];
                const int a = d.cur ^ parity;
                const View<P>& S = stage == 2 ? d.x : d.v[a];
                const View<P>& D = stage == 1 ? d.x : d.v[a ^ 1];
                boundary_newmark(d.g, d.c, S, D, d.bn, d.nb, S.s, d.tstep, bt.b);
            }
            continue;
        }
        if (tk.dom != cached) {
            __syncwarp();  // every lane is done with the previous descriptor
            const unsigned* src = reinterpret_cast<const unsigned*>(dd + tk.dom);
            unsigned* dst = reinterpret_cast<unsigned*>(sd + wid);
            for (int q = lane; q < (int)(sizeof(DomDesc<P>) / 4); q += 32) dst[q] = src[q];
            __syncwarp();
            cached = tk.dom;
        }
        const DomDesc<P>& d = sd[wid];
        const int a = d.cur ^ parity;
        bool bad;
        if (tk.kind == kPairStrip) {
            bad = pair_strip<P>(d.g, d.c, d.k, d.v[a], d.v[a ^ 1], tk.xs, tk.j0, tk.j1);
        } else {
            const View<P>& S = stage == 2 ? d.x : d.v[a];
            const View<P>& D = stage == 1 ? d.x : d.v[a ^ 1];
            bad = bulk_strip<P, 1, true>(d.g, d.c, d.k, S, D, tk.xs, tk.j0, tk.j1, Win{tk.x0, tk.x1, tk.y0, tk.y1});
        }
        if (__any_sync(FULL, bad) && lane == 0) atomicOr(d.flag, 1u);
    }
}

// ------------------------------------------------------------------ sync

// Sec. 3.2: phi, psi from differences of u at every point, populations by
// Eq. correction-f with the current first moments.  In place.
template <typename P>
__global__ void sync_kernel(Geo g, Consts c, KCof<P> k, View<P> A) {
    using V = typename P::V;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny || !body_at(g, i, j)) return;
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    size_t p = (size_t)j * g.px + i;
    double s[2];
    s[0] = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
    s[1] = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
    double jx[2], jy[2];
    for (int set = 0; set < 2; ++set) {
        V f[5];
        P::load5(A.f, g.plane, p, set, k, f);
        // first moments in the arithmetic type of the storage
        jx[set] = (double)sub_rn(f[1], f[3]);
        jy[set] = (double)sub_rn(f[2], f[4]);
    }
    P::store_eq_point(A.f, g.plane, p, c, s, jx, jy, k);
}

// ---------------------------------------------------------------- fields

template <typename P>
__device__ inline double moment0_fp64(const View<P>& A, size_t plane, size_t p, int set, const KCof<P>& k) {
    double b[5];
    P::load5d(A.f, plane, p, set, k, b);
    return b[0] + ((b[1] + b[2]) + (b[3] + b[4]));
}

// Scalar field value at (i, j).
template <typename P>
__device__ inline double field_value(const Geo& g, const Consts& c, const KCof<P>& k, const View<P>& A, int field,
                                     int i, int j) {
    size_t p = (size_t)j * g.px + i;
    switch (field) {
    case FLD_UX: case FLD_UY: case FLD_VX: case FLD_VY: return A.u[(size_t)field * g.plane + p];
    case FLD_PHI: return moment0_fp64(A, g.plane, p, 0, k);
    case FLD_PSI: return moment0_fp64(A, g.plane, p, 1, k);
    case FLD_KIN: {
        // kinetic energy density rho |du/dt|^2 / 2 (0 at void points)
        if (!body_at(g, i, j)) return 0.0;
        const double vx = A.u[2 * g.plane + p], vy = A.u[3 * g.plane + p];
        return 0.5 * c.rho * (vx * vx + vy * vy);
    }
    case FLD_STRAIN: {
        // strain energy density sigma : eps / 2 = lambda tr(eps)^2 / 2 + mu eps : eps
        // (Eq. hooke with eps of Eq. strain by the finite differences of Sec. 3.1.2)
        if (!body_at(g, i, j)) return 0.0;
        const double* ux = A.u;
        const double* uy = A.u + g.plane;
        const double exx = ddx(ux, g.px, i, j, g, c.inv2h);
        const double eyy = ddy(uy, g.px, i, j, g, c.inv2h);
        const double exy = 0.5 * (ddy(ux, g.px, i, j, g, c.inv2h) + ddx(uy, g.px, i, j, g, c.inv2h));
        const double tr = exx + eyy;
        return 0.5 * c.lam * tr * tr + c.mu * (exx * exx + eyy * eyy + 2.0 * exy * exy);
    }
    default: {
        // consistency error e(x, t) of Sec. 4 (0 at void points)
        if (!body_at(g, i, j)) return 0.0;
        const double* ux = A.u;
        const double* uy = A.u + g.plane;
        double div = ddx(ux, g.px, i, j, g, c.inv2h) + ddy(uy, g.px, i, j, g, c.inv2h);
        double curl = ddx(uy, g.px, i, j, g, c.inv2h) - ddy(ux, g.px, i, j, g, c.inv2h);
        double e1 = moment0_fp64(A, g.plane, p, 1, k) - curl;
        double e0 = moment0_fp64(A, g.plane, p, 0, k) - div;
        return sqrt(e1 * e1 + e0 * e0);
    }
    }
}

// Dense FP64 copy of rows [j0, j0 + rows) of a field.  Population fields
// write 5 consecutive [rows][nx] blocks.
template <typename P>
__global__ void extract_kernel(Geo g, Consts c, KCof<P> k, View<P> A, int field, int j0, int rows, double* dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int jr = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || jr >= rows) return;
    int j = j0 + jr;
    size_t d = (size_t)jr * g.nx + i;
    if (field == FLD_FPHI || field == FLD_FPSI) {
        int set = field == FLD_FPHI ? 0 : 1;
        size_t p = (size_t)j * g.px + i;
        size_t blk = (size_t)rows * g.nx;
        double f[5];
        P::load5d(A.f, g.plane, p, set, k, f);
        for (int q = 0; q < 5; ++q) dst[q * blk + d] = f[q];
        return;
    }
    dst[d] = field_value<P>(g, c, k, A, field, i, j);
}

// --------------------------------------------------------------- norms

constexpr int kNormThreads = 256;

template <typename P>
__global__ void __launch_bounds__(kNormThreads) norms_partial_kernel(Geo g, Consts c, KCof<P> k, View<P> A,
                                                                     int field,
                                                                     const double* __restrict__ ref,
                                                                     double* partials) {
    __shared__ double sh[4][kNormThreads];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, mx = 0.0;
    size_t n = (size_t)g.nx * g.ny;
    for (size_t d = (size_t)blockIdx.x * blockDim.x + threadIdx.x; d < n; d += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(d % g.nx), j = (int)(d / g.nx);
        double x = field_value<P>(g, c, k, A, field, i, j);
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

// Rows of a state copy to or from a caller buffer, 16 bytes per thread and
// step; segment blockIdx.y.  The lattice side of each copy goes through the
// checked accessors, the caller's buffer is not part of a lattice block.
__global__ void copy_segments_kernel(CopySegs s) {
    const int q = blockIdx.y;
    if (q >= s.n) return;
    const uint4* a = reinterpret_cast<const uint4*>(s.src[q]);
    uint4* b = reinterpret_cast<uint4*>(s.dst[q]);
    const size_t n16 = s.bytes[q] / 16;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n16; t += (size_t)gridDim.x * blockDim.x) {
#ifdef LBPS_CHECKED
        if (!chk_ok(s.pack ? &a[t] : &b[t], __LINE__)) continue;
#endif
        b[t] = a[t];
    }
}

dim3 grid2d(int nx, int ny, dim3 blk) { return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y); }

}  // namespace

// ------------------------------------------------------------- launchers

template <typename P>
cudaError_t launch_boundary_batch(const DomDesc<P>* dd, const BndTask* tasks, int ntasks, int parity, int pass_lo,
                                  int pass_hi, cudaStream_t st, int stage) {
    if (ntasks > 0)
        for (int pass = pass_lo; pass < pass_hi; ++pass) {
            boundary_batch_kernel<P><<<(ntasks + 127) / 128, 128, 0, st>>>(dd, tasks, ntasks, parity, pass, stage);
            if (pass == 2 && P::kSplitStream)
                boundary_batch_kernel<P><<<(ntasks + 127) / 128, 128, 0, st>>>(dd, tasks, ntasks, parity, 3, stage);
        }
    return cudaGetLastError();
}

// Blocks of the persistent batch kernel: those resident on all SMs at once.
template <typename K>
int resident_blocks(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * kWarpsPerBlock, 0) != cudaSuccess)
        return -1;
    return sms * (per_sm > 0 ? per_sm : 1);
}

template <typename P, int MINB, int UVD>
cudaError_t launch_bulk_batch_v(const DomDesc<P>* dd, const BulkTask* tasks, int ntasks, const BndTask* btasks,
                                int parity, unsigned* next, cudaStream_t st) {
    auto kern = bulk_batch_kernel<P, MINB, UVD>;
    int blocks = resident_blocks(kern);
    if (blocks < 0) return cudaGetLastError();
    blocks = min(blocks, (ntasks + kWarpsPerBlock - 1) / kWarpsPerBlock);
    cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(dd, tasks, ntasks, btasks, parity, next);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_pair_batch(const DomDesc<P>* dd, const PairTask* tasks, int ntasks, const BndTask* btasks,
                              int parity, int stage, unsigned* next, cudaStream_t st) {
    if (ntasks <= 0) return cudaGetLastError();
    // 4 blocks per SM (at 5 the two kinds of strips together spill)
    auto kern = pair_batch_kernel<P, sizeof(typename P::V) == 8 ? 2 : 4>;
    int blocks = resident_blocks(kern);
    if (blocks < 0) return cudaGetLastError();
    blocks = min(blocks, (ntasks + kWarpsPerBlock - 1) / kWarpsPerBlock);
    kern<<<blocks, 32 * kWarpsPerBlock, 0, st>>>(dd, tasks, ntasks, btasks, parity, stage, next);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_bulk_batch(const DomDesc<P>* dd, const BulkTask* tasks, int ntasks, const BndTask* btasks,
                              int parity, int variant, unsigned* next, cudaStream_t st) {
    if (ntasks <= 0) return cudaGetLastError();
    switch (variant) {
    case 0: return launch_bulk_batch_v<P, 6, 2>(dd, tasks, ntasks, btasks, parity, next, st);
    case 1: return launch_bulk_batch_v<P, 5, 2>(dd, tasks, ntasks, btasks, parity, next, st);
    case 2: return launch_bulk_batch_v<P, 4, 2>(dd, tasks, ntasks, btasks, parity, next, st);
    case 3: return launch_bulk_batch_v<P, 8, 2>(dd, tasks, ntasks, btasks, parity, next, st);
    case 4: return launch_bulk_batch_v<P, 6, 1>(dd, tasks, ntasks, btasks, parity, next, st);
    case 5: return launch_bulk_batch_v<P, 5, 1>(dd, tasks, ntasks, btasks, parity, next, st);
    case 6: return launch_bulk_batch_v<P, 4, 1>(dd, tasks, ntasks, btasks, parity, next, st);
    default: return launch_bulk_batch_v<P, 8, 1>(dd, tasks, ntasks, btasks, parity, next, st);
    }
}

cudaError_t launch_copy_segments(const CopySegs& s, cudaStream_t st) {
    if (s.n <= 0) return cudaSuccess;
    size_t most = 0;
    for (int q = 0; q < s.n; ++q) most = std::max(most, s.bytes[q] / 16);
    const int bx = (int)std::min<size_t>((most + 255) / 256, 1024);
    copy_segments_kernel<<<dim3(std::max(bx, 1), s.n), 256, 0, st>>>(s);
    return cudaGetLastError();
}

cudaError_t set_check_range(const void* base, size_t bytes, cudaStream_t st) {
#ifdef LBPS_CHECKED
    // the table of live blocks, mirrored on the host and uploaded whole
    static std::vector<std::pair<const char*, const char*>> ranges;
    const char* lo = static_cast<const char*>(base);
    ranges.erase(std::remove_if(ranges.begin(), ranges.end(), [&](const auto& r) { return r.first == lo; }),
                 ranges.end());
    if (bytes > 0) {
        if (ranges.size() >= (size_t)kChkRanges) return cudaErrorInvalidValue;
        ranges.emplace_back(lo, lo + bytes);
    }
    std::vector<const char*> los, his;
    for (const auto& r : ranges) {
        los.push_back(r.first);
        his.push_back(r.second);
    }
    const int n = (int)ranges.size();
    cudaError_t e = cudaStreamSynchronize(st);  // no kernel in flight sees a half-written table
    if (e == cudaSuccess && n > 0) e = cudaMemcpyToSymbol(g_chk_lo, los.data(), n * sizeof(const char*));
    if (e == cudaSuccess && n > 0) e = cudaMemcpyToSymbol(g_chk_hi, his.data(), n * sizeof(const char*));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_chk_n, &n, sizeof(n));
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

cudaError_t launch_finite_check(const Geo& g, const double* u, int planes, unsigned* bad, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return cudaGetLastError();
    const size_t total = (size_t)g.nx * (size_t)g.ny * (size_t)planes;
    const size_t want = (total + 255) / 256;
    const int blocks = (int)std::min<size_t>(want, (size_t)sms * 8);
    finite_check_kernel<<<blocks, 256, 0, st>>>(g, u, planes, bad);
    return cudaGetLastError();
}

cudaError_t launch_scale_probe(const Geo& g, const Consts& c, const double* u, double sq, unsigned* out,
                               cudaStream_t st) {
    dim3 blk(32, 8);
    scale_probe_kernel<<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, u, sq, out);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_init(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, cudaStream_t st) {
    dim3 blk(32, 8);
    init_kernel<P><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, k, A);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_mirror(const Geo& g, View<P> A, const BNode* bn, int nb, cudaStream_t st) {
    if (nb > 0) boundary_mirror_kernel<P><<<(nb + 127) / 128, 128, 0, st>>>(g, A, bn, nb);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_boundary(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, const BNode* bn,
                            int nb, unsigned* flag, unsigned long long* tstep, cudaStream_t st,
                            int pass_lo, int pass_hi) {
    if (nb > 0) {
        const int blocks = (nb + 127) / 128;
        for (int pass = pass_lo; pass < pass_hi; ++pass) {
            if (pass == 0) boundary_stress_kernel<P><<<blocks, 128, 0, st>>>(g, c, A, bn, nb);
            if (pass == 1) boundary_newmark_kernel<P><<<blocks, 128, 0, st>>>(g, c, A, B, bn, nb, tstep);
            if (pass == 2) boundary_reset_kernel<P><<<blocks, 128, 0, st>>>(g, c, k, A, B, bn, nb, flag, tstep);
            if (pass == 2 && P::kSplitStream)
                boundary_stream_y_kernel<P><<<blocks, 128, 0, st>>>(g, c, k, A, B, bn, nb);
        }
    }
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_bulk(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                        cudaStream_t st, const Tuning& tu) {
    int warps = (g.nx + kStripCols - 1) / kStripCols;
    dim3 grid((warps + kWarpsPerBlock - 1) / kWarpsPerBlock, (g.ny + tu.rows_per_warp - 1) / tu.rows_per_warp);
    dim3 blk(32 * kWarpsPerBlock);
    switch (tu.variant) {
    case 0: bulk_kernel<P, 6, 2><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 1: bulk_kernel<P, 5, 2><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 2: bulk_kernel<P, 4, 2><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 3: bulk_kernel<P, 8, 2><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 4: bulk_kernel<P, 6, 1><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 5: bulk_kernel<P, 5, 1><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    case 6: bulk_kernel<P, 4, 1><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    default: bulk_kernel<P, 8, 1><<<grid, blk, 0, st>>>(g, c, k, A, B, flag, tu.rows_per_warp); break;
    }
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_frame(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                         cudaStream_t st, int fw) {
    // FP64 populations need the 4-blocks shape (the others spill there);
    // BFP13 fits 6 blocks with u prefetched one row ahead, not two
    constexpr int minb = sizeof(typename P::V) == 8 ? 4 : 6;
    constexpr int uvd = std::is_same<P, PopBfp13>::value ? 1 : 2;
    auto kern = frame_kernel<P, minb, uvd>;
    const int nx = g.nx, ny = g.ny, rows = 32;
    const int all = (nx + kStripCols - 1) / kStripCols;
    const dim3 blk(32 * kWarpsPerBlock);
    auto blocks = [](int strips) { return (strips + kWarpsPerBlock - 1) / kWarpsPerBlock; };
    // top and bottom bands: every strip, fw rows
    kern<<<dim3(blocks(all), 1), blk, 0, st>>>(g, c, k, A, B, flag, 0, all, 1, 1 + fw, fw,
                                                Win{1, nx - 1, 1, 1 + fw});
    kern<<<dim3(blocks(all), 1), blk, 0, st>>>(g, c, k, A, B, flag, 0, all, ny - 1 - fw, ny - 1, fw,
                                                Win{1, nx - 1, ny - 1 - fw, ny - 1});
    // left and right bands between them: the strips holding columns 1 .. fw and
    // nx - 1 - fw .. nx - 2
    const int jb = 1 + fw, je = ny - 1 - fw, chunks = (je - jb + rows - 1) / rows;
    const int ls0 = 1 / kStripCols, ls1 = fw / kStripCols;
    const int rs0 = (nx - 1 - fw) / kStripCols, rs1 = (nx - 2) / kStripCols;
    kern<<<dim3(blocks(ls1 - ls0 + 1), chunks), blk, 0, st>>>(g, c, k, A, B, flag, ls0, ls1 - ls0 + 1, jb, je, rows,
                                                             Win{1, 1 + fw, jb, je});
    kern<<<dim3(blocks(rs1 - rs0 + 1), chunks), blk, 0, st>>>(g, c, k, A, B, flag, rs0, rs1 - rs0 + 1, jb, je, rows,
                                                             Win{nx - 1 - fw, nx - 1, jb, je});
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_pair(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                        cudaStream_t st, int rows) {
    const int warps = (g.nx - 2 * kDeep + kPairCols - 1) / kPairCols;
    const dim3 grid((warps + kWarpsPerBlock - 1) / kWarpsPerBlock, (g.ny - 2 * kDeep + rows - 1) / rows);
    // blocks per SM that fit without spilling: 5 for FP32 and the 16-bit
    // formats (96 registers; 8192^2 FP32: 70.2 against 67.1 GLUPS at 4),
    // 2 for FP64
    constexpr int minb = sizeof(typename P::V) == 8 ? 2 : 5;
    pair_kernel<P, minb><<<grid, 32 * kWarpsPerBlock, 0, st>>>(g, c, k, A, B, flag, rows);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_sync(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, cudaStream_t st) {
    dim3 blk(32, 8);
    sync_kernel<P><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, k, A);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_extract_rows(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, int field, int j0,
                                int rows, double* dst, cudaStream_t st) {
    dim3 blk(32, 8);
    extract_kernel<P><<<grid2d(g.nx, rows, blk), blk, 0, st>>>(g, c, k, A, field, j0, rows, dst);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_norms(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, int field, const double* ref,
                         double* partials, double* out4, cudaStream_t st) {
    size_t n = (size_t)g.nx * g.ny;
    int nblk = (int)((n + kNormThreads - 1) / kNormThreads);
    if (nblk > kNormBlocks) nblk = kNormBlocks;
    norms_partial_kernel<P><<<nblk, kNormThreads, 0, st>>>(g, c, k, A, field, ref, partials);
    norms_final_kernel<<<1, kNormThreads, 0, st>>>(partials, nblk, out4);
    return cudaGetLastError();
}

#define LBPS_INSTANTIATE(P)                                                                                   \
    template cudaError_t launch_init<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, cudaStream_t);  \
    template cudaError_t launch_frame<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, View<P>, unsigned*,  \
                                         cudaStream_t, int);                                                  \
    template cudaError_t launch_pair<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, View<P>, unsigned*,   \
                                        cudaStream_t, int);                                                   \
    template cudaError_t launch_mirror<P>(const Geo&, View<P>, const BNode*, int, cudaStream_t);            \
    template cudaError_t launch_boundary<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, View<P>,      \
                                            const BNode*, int, unsigned*, unsigned long long*,                \
                                            cudaStream_t, int, int);                                          \
    template cudaError_t launch_bulk<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, View<P>,          \
                                        unsigned*, cudaStream_t, const Tuning&);                              \
    template cudaError_t launch_sync<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, cudaStream_t);  \
    template cudaError_t launch_extract_rows<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, int, int, \
                                                int, double*, cudaStream_t);                                  \
    template cudaError_t launch_norms<P>(const Geo&, const Consts&, const KCof<P>&, View<P>, int,            \
                                         const double*, double*, double*, cudaStream_t);                     \
    template cudaError_t launch_boundary_batch<P>(const DomDesc<P>*, const BndTask*, int, int, int, int,      \
                                                  cudaStream_t, int);                                         \
    template cudaError_t launch_pair_batch<P>(const DomDesc<P>*, const PairTask*, int, const BndTask*, int, int, \
                                              unsigned*, cudaStream_t);                                       \
    template cudaError_t launch_bulk_batch<P>(const DomDesc<P>*, const BulkTask*, int, const BndTask*, int, int, \
                                              unsigned*, cudaStream_t);

LBPS_INSTANTIATE(PopDirect<float>)
LBPS_INSTANTIATE(PopDirect<double>)
LBPS_INSTANTIATE(PopNeq16<__nv_bfloat16>)
LBPS_INSTANTIATE(PopNeq16<__half>)
LBPS_INSTANTIATE(PopBfp13)

}  // namespace lbps
