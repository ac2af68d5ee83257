// Device-side types and shared device functions of the plane-strain LBM
// (arXiv:2301.00228).  Included by the kernel and ABI translation units only.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbps {

// Global-memory accessors of the kernels.  In a build with LBPS_CHECKED
// defined, every access is checked against the lattice's device block and
// for alignment; the first violation is recorded (source line and address)
// and the access is skipped, so a bad index shows up as a report instead of
// a fault.  Without LBPS_CHECKED they are plain loads and stores.
#ifdef LBPS_CHECKED
__device__ const char* g_chk_lo;
__device__ const char* g_chk_hi;
__device__ unsigned long long g_chk_line;
__device__ unsigned long long g_chk_addr;
template <typename P>
__device__ __forceinline__ bool chk_ok(const P* p, int line) {
    const char* c = reinterpret_cast<const char*>(p);
    bool ok = c >= g_chk_lo && c + sizeof(P) <= g_chk_hi && (reinterpret_cast<uintptr_t>(c) % sizeof(P)) == 0;
    if (!ok && atomicCAS(&g_chk_line, 0ull, (unsigned long long)line) == 0ull)
        g_chk_addr = reinterpret_cast<unsigned long long>(c);
    return ok;
}
#define LBPS_LDG(p) (::lbps::chk_ok((p), __LINE__) ? __ldg(p) : decltype(__ldg(p))(0))
#define LBPS_LD(p) (::lbps::chk_ok((p), __LINE__) ? *(p) : decltype(+*(p))(0))
#define LBPS_ST(p, v)                                      \
    do {                                                  \
        if (::lbps::chk_ok((p), __LINE__)) *(p) = (v);    \
    } while (0)
#else
#define LBPS_LDG(p) __ldg(p)
#define LBPS_LD(p) (*(p))
#define LBPS_ST(p, v) (*(p) = (v))
#endif

// Lattice geometry.  Planes are pitched: row j of a plane starts at j * px.
struct Geo {
    int nx, ny;
    int px;              // row pitch in elements (multiple of 32)
    int periodic_x, periodic_y;
    size_t plane;        // px * ny elements per plane
};

// FP64 constants of the method (Eq. conditions-parameters, Eq. integration).
struct Consts {
    double dt, half_dt2;        // Delta t, Delta t^2 / 2
    double lam, mu, rho, dh;
    double inv2h;               // 1 / (2 dh)
    double cd2, cs2;            // c_d^2, c_s^2 (c_s = sqrt(mu/rho))
    double a[2], a0[2];         // a_phi, a_psi ; a_{0,phi}, a_{0,psi}
    double two_dt2, two_dt;     // 2 / dt^2, 2 / dt (Eq. acc_dirichlet)
    double inv_rho_dh2;         // 1 / (rho dh^2); a boundary cell's 1 / (rho V_C) is 1, 2 or 4 times it
    int bc_feq_mode;            // Eq. LBE_mod reading
};

// The same constants in the population arithmetic type T.
template <typename T>
struct KC {
    T a[2];                     // weight of the moving populations
    T two_a[2];                 // 2 a
    T two_a0[2];                // 2 a_0
    T eight_a[2];               // 8 a = 2 (1 - a_0)
    T cd2h, cs2h;               // c_d^2 / (2 dh), c_s^2 / (2 dh)
};

// One state copy: 10 population planes (phi^0..phi^4, psi^0..psi^4) of type T
// and 4 FP64 planes (u_x, u_y, v_x, v_y).
template <typename T>
struct View {
    T* f;
    double* u;
};

// A boundary lattice point (perimeter order, see perim_index).
struct BNode {
    int i, j;
    int type;        // 1 Neumann, 2 Dirichlet
    int pad;
    double bx, by;   // u* (Dirichlet) or integrated external force (Neumann)
};

enum { NEUMANN = 1, DIRICHLET = 2 };

__host__ __device__ inline bool is_boundary(int i, int j, const Geo& g) {
    return (!g.periodic_x && (i == 0 || i == g.nx - 1)) || (!g.periodic_y && (j == 0 || j == g.ny - 1));
}

// Position of boundary point (i, j) in the perimeter list: bottom row, top
// row (when y is bounded), then left and right columns without the corners.
__host__ __device__ inline int perim_index(int i, int j, const Geo& g) {
    int rows = g.periodic_y ? 0 : 2 * g.nx;
    if (!g.periodic_y) {
        if (j == 0) return i;
        if (j == g.ny - 1) return g.nx + i;
    }
    int jlo = g.periodic_y ? 0 : 1;
    int collen = g.periodic_y ? g.ny : g.ny - 2;
    if (i == 0) return rows + (j - jlo);
    return rows + collen + (j - jlo);
}

__host__ __device__ inline int perim_count(const Geo& g) {
    int rows = g.periodic_y ? 0 : 2 * g.nx;
    int collen = g.periodic_y ? g.ny : g.ny - 2;
    int cols = g.periodic_x ? 0 : 2 * collen;
    return rows + cols;
}

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Explicitly rounded arithmetic so every kernel that evaluates a shared
// formula produces the same bits (no compiler-chosen contraction).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// One-dimensional second-order difference stencil at index i of n points:
// central where both neighbours exist (or wrap), one-sided three-point at a
// non-periodic end.  Offsets and weights (to be scaled by 1/(2 dh)).
struct Sten {
    int n;
    int d[3];
    double w[3];
};

__device__ __forceinline__ Sten stencil(int i, int n, int periodic) {
    Sten s;
    if (periodic || (i > 0 && i < n - 1)) {
        s.n = 2; s.d[0] = -1; s.w[0] = -1.0; s.d[1] = 1; s.w[1] = 1.0; s.d[2] = 0; s.w[2] = 0.0;
    } else if (i == 0) {
        s.n = 3; s.d[0] = 0; s.w[0] = -3.0; s.d[1] = 1; s.w[1] = 4.0; s.d[2] = 2; s.w[2] = -1.0;
    } else {
        s.n = 3; s.d[0] = 0; s.w[0] = 3.0; s.d[1] = -1; s.w[1] = -4.0; s.d[2] = -2; s.w[2] = 1.0;
    }
    return s;
}

// d/dx and d/dy of a FP64 array with row stride `stride` (reading of the
// paper's "second order accurate finite differences", Sec. 3.1.2).
__device__ inline double ddx(const double* __restrict__ g, size_t stride, int i, int j, const Geo& G,
                             double inv2h) {
    Sten s = stencil(i, G.nx, G.periodic_x);
    const double* r = g + (size_t)j * stride;
    double acc = 0.0;
    for (int q = 0; q < s.n; ++q) acc = fma_rn(s.w[q], LBPS_LD(&r[wrap(i + s.d[q], G.nx)]), acc);
    return mul_rn(acc, inv2h);
}

__device__ inline double ddy(const double* __restrict__ g, size_t stride, int i, int j, const Geo& G,
                             double inv2h) {
    Sten s = stencil(j, G.ny, G.periodic_y);
    double acc = 0.0;
    for (int q = 0; q < s.n; ++q) acc = fma_rn(s.w[q], LBPS_LD(&g[(size_t)wrap(j + s.d[q], G.ny) * stride + i]), acc);
    return mul_rn(acc, inv2h);
}

// Interior acceleration, Eq. navier: a = c_d^2 grad(phi) - c_s^2 curl(psi e_z)
// with central differences of the neighbours' moments.  Evaluated in the
// population type T and widened to FP64 for the Newmark update.
template <typename T>
__device__ __forceinline__ void accel_interior(T phiW, T phiE, T phiS, T phiN, T psiW, T psiE, T psiS,
                                               T psiN, const KC<T>& k, double& ax, double& ay) {
    T dphix = sub_rn(phiE, phiW), dphiy = sub_rn(phiN, phiS);
    T dpsix = sub_rn(psiE, psiW), dpsiy = sub_rn(psiN, psiS);
    ax = (double)fma_rn(k.cd2h, dphix, -mul_rn(k.cs2h, dpsiy));
    ay = (double)fma_rn(k.cd2h, dphiy, mul_rn(k.cs2h, dpsix));
}

// Eq. integration (explicit Newmark as printed).
__device__ __forceinline__ void newmark(double u, double v, double a, const Consts& c, double& u1, double& v1) {
    u1 = fma_rn(c.half_dt2, a, fma_rn(c.dt, v, u));
    v1 = fma_rn(c.dt, a, v);
}

template <typename T>
__device__ __forceinline__ T sum5(T f0, T f1, T f2, T f3, T f4) {
    return add_rn(f0, add_rn(add_rn(f1, f2), add_rn(f3, f4)));
}

}  // namespace lbps
