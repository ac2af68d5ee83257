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
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

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
    b[0] = (T)(a0 * s);
    b[plane] = (T)(as + 0.5 * jx);
    b[2 * plane] = (T)(as + 0.5 * jy);
    b[3 * plane] = (T)(as - 0.5 * jx);
    b[4 * plane] = (T)(as - 0.5 * jy);
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
    double vx = A.u[2 * g.plane + p], vy = A.u[3 * g.plane + p];
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
// F = int t* da supplied per point.
__device__ inline void accel_neumann(const Geo& g, const Consts& c, const double* ux, const double* uy,
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
    stress_at(g, c, ux, uy, i, j, sk);
    for (int d = 0; d < 4; ++d) {
        if (!has[d]) continue;
        int ri = wrap(i + DX[d], g.nx), rj = wrap(j + DY[d], g.ny);
        double sr[3];
        stress_at(g, c, ux, uy, ri, rj, sr);
        double sxx = 0.5 * (sk[0] + sr[0]);
        double syy = 0.5 * (sk[1] + sr[1]);
        double sxy = 0.5 * (sk[2] + sr[2]);
        double len = DX[d] != 0 ? wy : wx;
        fx += (sxx * DX[d] + sxy * DY[d]) * len;
        fy += (sxy * DX[d] + syy * DY[d]) * len;
    }
    double m = c.rho * wx * wy;
    ax = fx / m;
    ay = fy / m;
}

// Acceleration at time t of any lattice point (interior: Eq. navier; boundary:
// Eq. acc_neumann or Eq. acc_dirichlet).
template <typename T>
__device__ inline void accel_at(const Geo& g, const Consts& c, const KC<T>& k, const View<T>& A,
                                const BNode* __restrict__ bn, int i, int j, double& ax, double& ay) {
    const double* ux = A.u;
    const double* uy = A.u + g.plane;
    size_t p = (size_t)j * g.px + i;
    if (is_boundary(i, j, g)) {
        BNode b = bn[perim_index(i, j, g)];
        if (b.type == DIRICHLET) {
            const double* vx = A.u + 2 * g.plane;
            const double* vy = A.u + 3 * g.plane;
            double two_dt2 = 2.0 / (c.dt * c.dt), two_dt = 2.0 / c.dt;
            ax = two_dt2 * (b.bx - ux[p]) - two_dt * vx[p];
            ay = two_dt2 * (b.by - uy[p]) - two_dt * vy[p];
        } else {
            accel_neumann(g, c, ux, uy, i, j, b.bx, b.by, ax, ay);
        }
        return;
    }
    int iw = wrap(i - 1, g.nx), ie = wrap(i + 1, g.nx), js = wrap(j - 1, g.ny), jn = wrap(j + 1, g.ny);
    size_t pw = (size_t)j * g.px + iw, pe = (size_t)j * g.px + ie;
    size_t ps = (size_t)js * g.px + i, pn = (size_t)jn * g.px + i;
    accel_interior<T>(moment0(A.f, g.plane, pw, 0), moment0(A.f, g.plane, pe, 0), moment0(A.f, g.plane, ps, 0),
                      moment0(A.f, g.plane, pn, 0), moment0(A.f, g.plane, pw, 1), moment0(A.f, g.plane, pe, 1),
                      moment0(A.f, g.plane, ps, 1), moment0(A.f, g.plane, pn, 1), k, ax, ay);
}

template <typename T>
__device__ inline void unew_at(const Geo& g, const Consts& c, const KC<T>& k, const View<T>& A,
                               const BNode* __restrict__ bn, int i, int j, double& ux1, double& uy1,
                               double& vx1, double& vy1) {
    double ax, ay;
    accel_at(g, c, k, A, bn, i, j, ax, ay);
    size_t p = (size_t)j * g.px + i;
    newmark(A.u[p], A.u[2 * g.plane + p], ax, c, ux1, vx1);
    newmark(A.u[g.plane + p], A.u[3 * g.plane + p], ay, c, uy1, vy1);
}

template <typename T>
__global__ void __launch_bounds__(128) boundary_kernel(Geo g, Consts c, KC<T> k, View<T> A, View<T> B,
                                                       const BNode* __restrict__ bn, int nb, unsigned* flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int i = bn[b].i, j = bn[b].j;
    size_t p = (size_t)j * g.px + i;
    double ux1, uy1, vx1, vy1;
    unew_at(g, c, k, A, bn, i, j, ux1, uy1, vx1, vy1);
    // Eq. psi_phi_at_bound: differences of u(t + dt) at (i, j).
    Sten sx = stencil(i, g.nx, g.periodic_x), sy = stencil(j, g.ny, g.periodic_y);
    double dux_dx = 0.0, duy_dx = 0.0, dux_dy = 0.0, duy_dy = 0.0;
    for (int q = 0; q < sx.n; ++q) {
        double a1 = ux1, a2 = uy1, t1, t2;
        if (sx.d[q] != 0) unew_at(g, c, k, A, bn, wrap(i + sx.d[q], g.nx), j, a1, a2, t1, t2);
        dux_dx = fma_rn(sx.w[q], a1, dux_dx);
        duy_dx = fma_rn(sx.w[q], a2, duy_dx);
    }
    for (int q = 0; q < sy.n; ++q) {
        double a1 = ux1, a2 = uy1, t1, t2;
        if (sy.d[q] != 0) unew_at(g, c, k, A, bn, i, wrap(j + sy.d[q], g.ny), a1, a2, t1, t2);
        dux_dy = fma_rn(sy.w[q], a1, dux_dy);
        duy_dy = fma_rn(sy.w[q], a2, duy_dy);
    }
    double phi = mul_rn(dux_dx, c.inv2h) + mul_rn(duy_dy, c.inv2h);
    double psi = mul_rn(duy_dx, c.inv2h) - mul_rn(dux_dy, c.inv2h);
    // Eq. correction-f with J(x_k, t) of the stored populations.
    for (int set = 0; set < 2; ++set) {
        const T* fa = A.f + (size_t)set * 5 * g.plane + p;
        double jx = (double)ld(fa + g.plane) - (double)ld(fa + 3 * g.plane);
        double jy = (double)ld(fa + 2 * g.plane) - (double)ld(fa + 4 * g.plane);
        store_feq(B.f, g.plane, p, set, c.a0[set], c.a[set], set == 0 ? phi : psi, jx, jy);
    }
    B.u[p] = ux1;
    B.u[g.plane + p] = uy1;
    B.u[2 * g.plane + p] = vx1;
    B.u[3 * g.plane + p] = vy1;
    if (!isfinite((T)phi + (T)psi)) atomicOr(flag, 1u);
}

// ---------------------------------------------------------------- bulk

// Value streamed out of a boundary source (Eq. LBE_mod).  f-hat is the mean
// of the stored (A) and reset (B) populations of the source; the
// equilibrium is taken from f-hat (mode 0) or from f(x_k, t) (mode 1).
// alpha is the direction of travel (1..4), opp its reverse.
template <typename T>
__device__ inline T stream_from_boundary(const T* __restrict__ fa, const T* __restrict__ fb, size_t plane,
                                         int alpha, int opp, const KC<T>& k, int set, int mode) {
    T a5[5], h5[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        a5[q] = ld(fa + q * plane);
        h5[q] = mul_rn((T)0.5, add_rn(a5[q], ld(fb + q * plane)));
    }
    if (mode == 0) {
        T sh = sum5(h5[0], h5[1], h5[2], h5[3], h5[4]);
        return fma_rn(k.two_a[set], sh, -h5[opp]);  // 2 f_eq(f-hat) - f-hat = 2 a s-hat - f-hat^opp
    }
    T sa = sum5(a5[0], a5[1], a5[2], a5[3], a5[4]);
    T ej = sub_rn(a5[alpha], a5[opp]);              // e_alpha . Jbar(x_k, t)
    return sub_rn(add_rn(mul_rn(k.two_a[set], sa), ej), h5[alpha]);
}

template <typename T>
__global__ void __launch_bounds__(256) bulk_kernel(Geo g, Consts c, KC<T> k, View<T> A, View<T> B,
                                                   unsigned* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    bool active = i < g.nx && j < g.ny && !is_boundary(i, j, g);
    bool bad = false;
    if (active) {
        int iw = wrap(i - 1, g.nx), ie = wrap(i + 1, g.nx), js = wrap(j - 1, g.ny), jn = wrap(j + 1, g.ny);
        size_t p = (size_t)j * g.px + i;
        size_t pw = (size_t)j * g.px + iw, pe = (size_t)j * g.px + ie;
        size_t ps = (size_t)js * g.px + i, pn = (size_t)jn * g.px + i;
        bool bw = is_boundary(iw, j, g), be = is_boundary(ie, j, g);
        bool bs = is_boundary(i, js, g), bnb = is_boundary(i, jn, g);
        T sW[2], sE[2], sS[2], sN[2];
        T out[2][5];
#pragma unroll
        for (int set = 0; set < 2; ++set) {
            const T* F = A.f + (size_t)set * 5 * g.plane;
            const T* FB = B.f + (size_t)set * 5 * g.plane;
            const size_t P = g.plane;
            // rest population: 2 a0 s - f0 = f0 + (2 a0 m - 8 a f0), m = moving sum
            T f0 = ld(F + p);
            T m = add_rn(add_rn(ld(F + P + p), ld(F + 2 * P + p)), add_rn(ld(F + 3 * P + p), ld(F + 4 * P + p)));
            out[set][0] = add_rn(f0, fma_rn(k.two_a0[set], m, -mul_rn(k.eight_a[set], f0)));
            // moving populations: f^alpha(x) = 2 a s(x - e_alpha) - f^opp(x - e_alpha)
            sW[set] = moment0(A.f, P, pw, set);
            sE[set] = moment0(A.f, P, pe, set);
            sS[set] = moment0(A.f, P, ps, set);
            sN[set] = moment0(A.f, P, pn, set);
            out[set][1] = bw ? stream_from_boundary(F + pw, FB + pw, P, 1, 3, k, set, c.bc_feq_mode)
                             : fma_rn(k.two_a[set], sW[set], -ld(F + 3 * P + pw));
            out[set][3] = be ? stream_from_boundary(F + pe, FB + pe, P, 3, 1, k, set, c.bc_feq_mode)
                             : fma_rn(k.two_a[set], sE[set], -ld(F + P + pe));
            out[set][2] = bs ? stream_from_boundary(F + ps, FB + ps, P, 2, 4, k, set, c.bc_feq_mode)
                             : fma_rn(k.two_a[set], sS[set], -ld(F + 4 * P + ps));
            out[set][4] = bnb ? stream_from_boundary(F + pn, FB + pn, P, 4, 2, k, set, c.bc_feq_mode)
                              : fma_rn(k.two_a[set], sN[set], -ld(F + 2 * P + pn));
        }
        double ax, ay;
        accel_interior<T>(sW[0], sE[0], sS[0], sN[0], sW[1], sE[1], sS[1], sN[1], k, ax, ay);
        double ux1, uy1, vx1, vy1;
        newmark(ld(A.u + p), ld(A.u + 2 * g.plane + p), ax, c, ux1, vx1);
        newmark(ld(A.u + g.plane + p), ld(A.u + 3 * g.plane + p), ay, c, uy1, vy1);
#pragma unroll
        for (int set = 0; set < 2; ++set)
#pragma unroll
            for (int q = 0; q < 5; ++q) B.f[((size_t)set * 5 + q) * g.plane + p] = out[set][q];
        B.u[p] = ux1;
        B.u[g.plane + p] = uy1;
        B.u[2 * g.plane + p] = vx1;
        B.u[3 * g.plane + p] = vy1;
        bad = !isfinite(out[0][0] + out[1][0]);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
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
cudaError_t launch_init(const Geo& g, const Consts& c, const KC<T>&, View<T> A, const double*, const double*,
                        const double*, const double*, cudaStream_t st) {
    dim3 blk(32, 8);
    init_kernel<T><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, A);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_boundary(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B, const BNode* bn,
                            int nb, unsigned* flag, cudaStream_t st) {
    if (nb > 0) boundary_kernel<T><<<(nb + 127) / 128, 128, 0, st>>>(g, c, k, A, B, bn, nb, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bulk(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B, unsigned* flag,
                        cudaStream_t st) {
    dim3 blk(32, 8);
    bulk_kernel<T><<<grid2d(g.nx, g.ny, blk), blk, 0, st>>>(g, c, k, A, B, flag);
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
                                            const BNode*, int, unsigned*, cudaStream_t);                      \
    template cudaError_t launch_bulk<T>(const Geo&, const Consts&, const KC<T>&, View<T>, View<T>, unsigned*, \
                                        cudaStream_t);                                                        \
    template cudaError_t launch_sync<T>(const Geo&, const Consts&, const KC<T>&, View<T>, cudaStream_t);     \
    template cudaError_t launch_extract<T>(const Geo&, const Consts&, View<T>, int, double*, cudaStream_t);  \
    template cudaError_t launch_extract_rows<T>(const Geo&, const Consts&, View<T>, int, int, int, double*,   \
                                                cudaStream_t);                                                \
    template cudaError_t launch_norms<T>(const Geo&, const Consts&, View<T>, int, const double*, double*,    \
                                         double*, cudaStream_t);

LBPS_INSTANTIATE(float)
LBPS_INSTANTIATE(double)

}  // namespace lbps
