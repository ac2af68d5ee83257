// Device-side types and shared device functions of the plane-strain LBM
// (arXiv:2301.00228).  Included by the kernel and ABI translation units only.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbps {

// Global-memory accessors of the kernels.  In a build with LBPS_CHECKED
// defined, every access is checked for alignment and against the device
// blocks of the live lattices (a table of at most kChkRanges); the first
// violation since the library was loaded is recorded (source line and
// address) and the access is skipped, so a bad index shows up as a report
// instead of a fault.  Without LBPS_CHECKED they are plain loads and stores.
#ifdef LBPS_CHECKED
constexpr int kChkRanges = 1024;
__device__ const char* g_chk_lo[kChkRanges];
__device__ const char* g_chk_hi[kChkRanges];
__device__ int g_chk_n;
__device__ unsigned long long g_chk_line;
__device__ unsigned long long g_chk_addr;
template <typename P>
__device__ __forceinline__ bool chk_ok(const P* p, int line) {
    const char* c = reinterpret_cast<const char*>(p);
    bool ok = (reinterpret_cast<uintptr_t>(c) % sizeof(P)) == 0;
    if (ok) {
        ok = false;
        for (int q = 0; q < g_chk_n && !ok; ++q) ok = c >= g_chk_lo[q] && c + sizeof(P) <= g_chk_hi[q];
    }
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
// general = 0: a rectangle whose boundary points are its outer ring (node
// classes from the indices).  general = 1: node types from the plane `type`
// (0 interior, 1 Neumann, 2 Dirichlet, 3 void), cells given per boundary
// point (reading R14: a plate with a hole).
struct Geo {
    int nx, ny;
    int px;              // row pitch in elements (multiple of 32)
    int periodic_x, periodic_y;
    int general;
    size_t plane;        // px * ny elements per plane
    const uint8_t* type; // [ny][px] node types (general = 1 only)
    size_t mplane;       // plane of the boundary mirror (boundary points, rounded up to 32)
    // general geometry: per 30-column strip s of the interior kernel, gap[2s]
    // .. gap[2s + 1] is the longest run of rows in which none of the strip's
    // columns holds an interior point (empty run: 0, 0); null for rectangles
    const int* gap;
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
    double load_rate[2];        // 1 / t_ramp of the Neumann [0] / Dirichlet [1] data (0: constant)
    double load_hold[2];        // t_hold: the factor is min(t, t_hold) / t_ramp
    int bc_feq_mode;            // Eq. LBE_mod reading
    int bc_j_mode;              // J of Eq. correction-f: 0 stored, 1 partial LBE update
};

// Time factor of the boundary data of one kind (0 Neumann, 1 Dirichlet) at
// time t: ramp then hold, 1 without a schedule (Sec. 4 loads).
__device__ __forceinline__ double load_factor(const Consts& c, int kind, double t) {
    return c.load_rate[kind] > 0.0 ? c.load_rate[kind] * fmin(t, c.load_hold[kind]) : 1.0;
}

// The same constants in the population arithmetic type T.
template <typename T>
struct KC {
    T a[2];                     // weight of the moving populations
    T two_a[2];                 // 2 a
    T two_a0[2];                // 2 a_0
    T eight_a[2];               // 8 a = 2 (1 - a_0)
    T cd2h, cs2h;               // c_d^2 / (2 dh), c_s^2 / (2 dh)
    T r[2];                     // a / a_0 (16-bit storage: equilibrium pair sum 2 r f^0)
    T scale, inv_scale;         // 2^e, 2^-e applied to the stored 16-bit Nx, Ny
    unsigned sr;                // 16-bit storage: round the stored sums stochastically (f2bits_store)
    unsigned key4;              // 4 x the offset added to a point's plane offset to form its
                                // rounding key (a sub-lattice of a larger one sets its first
                                // row's offset there)
};

// One state copy: the population planes (layout set by the storage policy P),
// 4 FP64 planes (u_x, u_y, v_x, v_y), and the boundary mirror: the
// populations of the boundary points again, in the order of the boundary
// list (planes of Geo::mplane points, same policy layout), so that the
// boundary reset reads and writes them coalesced; and the stresses of this
// copy's u that Eq. acc_neumann reads (3 doubles per slot: 2 slots per
// boundary point of a rectangle, 5 of a general geometry).
template <typename P>
struct View {
    typename P::Base* f;
    double* u;
    typename P::Base* m;
    double* s;
};

// A boundary lattice point (perimeter order, see perim_index).
struct BNode {
    int i, j;
    int type;        // 1 Neumann, 2 Dirichlet
    int smask;       // bit d: the neighbour in direction d (E, N, W, S) is interior (Eq. LBE_mod target)
    double bx, by;   // u* (Dirichlet) or integrated external force (Neumann)
    double inv_m;    // 1 / (rho V_C) of the cell (general geometry)
    double l[4];     // in-body lengths of the cell's sides E, N, W, S (general geometry)
    int nbmask;      // bit d: the neighbour in direction d is in the body (general geometry)
    int pad;
};

enum { NEUMANN = 1, DIRICHLET = 2, VOID = 3 };

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

// Is (i, j) (wrapped along periodic axes) a point of the body?
__device__ __forceinline__ bool body_at(const Geo& g, int i, int j) {
    if (i < 0 || i >= g.nx) {
        if (!g.periodic_x) return false;
        i = wrap(i, g.nx);
    }
    if (j < 0 || j >= g.ny) {
        if (!g.periodic_y) return false;
        j = wrap(j, g.ny);
    }
    return !g.general || LBPS_LDG(&g.type[(size_t)j * g.px + i]) != VOID;
}

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

// The same choice from the node types (general geometry, reading R14):
// central where both neighbours along (dx, dy) are in the body, else
// one-sided towards the body (its existence is checked at creation).
__device__ __forceinline__ Sten stencil_g(const Geo& g, int i, int j, int dx, int dy) {
    Sten s;
    const bool hp = body_at(g, i + dx, j + dy), hm = body_at(g, i - dx, j - dy);
    if (hp && hm) {
        s.n = 2; s.d[0] = -1; s.w[0] = -1.0; s.d[1] = 1; s.w[1] = 1.0; s.d[2] = 0; s.w[2] = 0.0;
    } else if (hp) {
        s.n = 3; s.d[0] = 0; s.w[0] = -3.0; s.d[1] = 1; s.w[1] = 4.0; s.d[2] = 2; s.w[2] = -1.0;
    } else {
        s.n = 3; s.d[0] = 0; s.w[0] = 3.0; s.d[1] = -1; s.w[1] = -4.0; s.d[2] = -2; s.w[2] = 1.0;
    }
    return s;
}

__device__ __forceinline__ Sten stencil_x(const Geo& G, int i, int j) {
    return G.general ? stencil_g(G, i, j, 1, 0) : stencil(i, G.nx, G.periodic_x);
}
__device__ __forceinline__ Sten stencil_y(const Geo& G, int i, int j) {
    return G.general ? stencil_g(G, i, j, 0, 1) : stencil(j, G.ny, G.periodic_y);
}

// d/dx and d/dy of a FP64 array with row stride `stride` (reading of the
// paper's "second order accurate finite differences", Sec. 3.1.2).
// (A central difference, weights -1 and 1, is one subtraction: the same
// bits as the weighted sum, fewer FP64 operations.)
__device__ inline double ddx(const double* __restrict__ g, size_t stride, int i, int j, const Geo& G,
                             double inv2h) {
    Sten s = stencil_x(G, i, j);
    const double* r = g + (size_t)j * stride;
    double acc = 0.0;
    if (s.n == 2)
        acc = sub_rn(LBPS_LD(&r[wrap(i + 1, G.nx)]), LBPS_LD(&r[wrap(i - 1, G.nx)]));
    else
        for (int q = 0; q < s.n; ++q) acc = fma_rn(s.w[q], LBPS_LD(&r[wrap(i + s.d[q], G.nx)]), acc);
    return mul_rn(acc, inv2h);
}

__device__ inline double ddy(const double* __restrict__ g, size_t stride, int i, int j, const Geo& G,
                             double inv2h) {
    Sten s = stencil_y(G, i, j);
    double acc = 0.0;
    if (s.n == 2)
        acc = sub_rn(LBPS_LD(&g[(size_t)wrap(j + 1, G.ny) * stride + i]),
                     LBPS_LD(&g[(size_t)wrap(j - 1, G.ny) * stride + i]));
    else
        for (int q = 0; q < s.n; ++q)
            acc = fma_rn(s.w[q], LBPS_LD(&g[(size_t)wrap(j + s.d[q], G.ny) * stride + i]), acc);
    return mul_rn(acc, inv2h);
}

// Interior acceleration, Eq. navier: a = c_d^2 grad(phi) - c_s^2 curl(psi e_z)
// with central differences of the neighbours' moments.  Evaluated in the
// population type T and widened to FP64 for the Newmark update.
template <typename T>
__device__ __forceinline__ void accel_interior_v(T phiW, T phiE, T phiS, T phiN, T psiW, T psiE, T psiS,
                                                 T psiN, const KC<T>& k, T& ax, T& ay) {
    T dphix = sub_rn(phiE, phiW), dphiy = sub_rn(phiN, phiS);
    T dpsix = sub_rn(psiE, psiW), dpsiy = sub_rn(psiN, psiS);
    ax = fma_rn(k.cd2h, dphix, -mul_rn(k.cs2h, dpsiy));
    ay = fma_rn(k.cd2h, dphiy, mul_rn(k.cs2h, dpsix));
}
template <typename T>
__device__ __forceinline__ void accel_interior(T phiW, T phiE, T phiS, T phiN, T psiW, T psiE, T psiS,
                                               T psiN, const KC<T>& k, double& ax, double& ay) {
    T x, y;
    accel_interior_v<T>(phiW, phiE, phiS, phiN, psiW, psiE, psiS, psiN, k, x, y);
    ax = (double)x;
    ay = (double)y;
}

// Eq. integration (explicit Newmark as printed).
__device__ __forceinline__ void newmark(double u, double v, double a, const Consts& c, double& u1, double& v1) {
    u1 = fma_rn(c.half_dt2, a, fma_rn(c.dt, v, u));
    v1 = fma_rn(c.dt, a, v);
}

// Two steps of Eq. integration at once, from the accelerations a0 at t and
// a1 at t + dt: u(t + 2 dt) = u + 2 dt v + dt^2/2 (3 a0 + a1) and
// v(t + 2 dt) = v + dt (a0 + a1), the two explicit updates composed.  The
// sums of the accelerations are taken in their own type (FP32 for the FP32
// and 16-bit storages, as the accelerations themselves), so u and v take 3
// FP64 fused multiply-adds each instead of 6; they differ from two calls of
// newmark by rounding only.
// FP32 -> FP64 exactly by integer operations only (the conversion
// instruction runs on the FP64 pipe, which the update keeps busy): the
// binary32 sign, exponent and fraction placed in binary64's fields.  Normal
// numbers: exponent rebased from 127 to 1023, fraction shifted up 29 bits.
// Zero: zero.  Subnormals m 2^-149 (m < 2^23, leading one at bit k):
// exponent k - 149 + 1023, the bits below the leading one as the fraction.
// Infinity and NaN: exponent 2047, the fraction (a NaN's payload) kept.
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu, E;
    if (e == 255u) {
        E = 2047u;
    } else if (e != 0u) {
        E = e + 896u;
    } else if (m != 0u) {
        const unsigned k = 31u - (unsigned)__clz(m);   // bit of the leading one, 0..22
        E = k + 874u;
        m = (m << (23u - k)) & 0x7fffffu;
    } else {
        E = 0u;
    }
    const unsigned hi = (u & 0x80000000u) | (E << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}

template <typename T>
__device__ __forceinline__ void newmark2(double u, double v, T a0, T a1, const Consts& c, double& u2, double& v2) {
    const double sa = widen(fma_rn((T)3, a0, a1)), sb = widen(add_rn(a0, a1));
    u2 = fma_rn(c.half_dt2, sa, fma_rn(c.dt + c.dt, v, u));
    v2 = fma_rn(c.dt, sb, v);
}

template <typename T>
__device__ __forceinline__ T sum5(T f0, T f1, T f2, T f3, T f4) {
    return add_rn(f0, add_rn(add_rn(f1, f2), add_rn(f3, f4)));
}

// ---- population storage policies
//
// PopDirect<T>: the five populations of each set as 10 planes of T (FP32 or
// FP64), arithmetic in T.
// PopNeq16<H>: per set the conserved moments in FP32 and the non-equilibrium
// part in 16 bits (H = __half or __nv_bfloat16), arithmetic in FP32.  The
// five populations of a set map one-to-one to f^0, the lattice first moment
// (Jx, Jy) = (f^1 - f^3, f^2 - f^4) and the pair sums f^1 + f^3, f^2 + f^4;
// at equilibrium (Eq. feq) each pair sum is 2 a s = 2 (a / a_0) f^0, so
//   Nx = f^1 + f^3 - 2 r f^0,  Ny = f^2 + f^4 - 2 r f^0   (r = a / a_0)
// vanish there and carry only the non-equilibrium part.  f^0, Jx, Jy are
// stored in FP32, Nx, Ny in H multiplied by 2^e (rounded by
// f2bits_store: to nearest, or stochastically with a_0 near 1).  Decoding:
//   f^1 = r f^0 + (Nx + Jx) / 2,  f^3 = r f^0 + (Nx - Jx) / 2  (and y).
// The first moment stays FP32 because with the small time steps of Sec. 4
// (a_0 near 1) every rounding of J acts as a momentum kick whose effect on
// phi grows with time; the pair sums do not have that effect.  Layout per
// copy: f^0, Jx, Jy of phi, the same of psi (6 FP32 planes), then two planes
// of 32-bit words, (Nx of phi | Nx of psi << 16) and the same for Ny, so every
// access is a 4-byte one; 32 bytes per point instead of 40.
//
// Besides per-set loads and stores, each policy writes a whole point
// (store_point, both sets) and one streamed population of both sets
// (store1_both), the forms the interior kernel and the boundary reset use.

template <typename T>
struct PopDirect {
    using V = T;
    using Base = T;
    static constexpr int kBytesPerPoint = 10 * (int)sizeof(T);
    // false: the boundary reset may write the x pair and the y pair of one
    // point from two threads at once (true for PopBfp13, whose words hold both)
    static constexpr bool kSplitStream = false;
    struct Raw {
        T f[2][5];
    };
    __device__ __forceinline__ static void load_raw(const T* __restrict__ f, size_t plane, size_t p, bool ok,
                                                    Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 5; ++q) r.f[s][q] = ok ? LBPS_LDG(f + (size_t)(s * 5 + q) * plane + p) : (T)0;
    }
    __device__ __forceinline__ static void decode(const Raw& r, int s, const KC<T>&, T (&x)[5]) {
#pragma unroll
        for (int q = 0; q < 5; ++q) x[q] = r.f[s][q];
    }
    __device__ __forceinline__ static void load5(const T* __restrict__ f, size_t plane, size_t p, int s,
                                                 const KC<T>&, T (&x)[5]) {
#pragma unroll
        for (int q = 0; q < 5; ++q) x[q] = LBPS_LD(f + (size_t)(s * 5 + q) * plane + p);
    }
    __device__ __forceinline__ static void store5(T* __restrict__ f, size_t plane, size_t p, int s, const T (&x)[5],
                                                  const KC<T>&) {
#pragma unroll
        for (int q = 0; q < 5; ++q) LBPS_ST(f + (size_t)(s * 5 + q) * plane + p, x[q]);
    }
    __device__ __forceinline__ static void store_point(T* __restrict__ f, size_t plane, size_t p,
                                                       const T (&x)[2][5], const KC<T>& k) {
#pragma unroll
        for (int s = 0; s < 2; ++s) store5(f, plane, p, s, x[s], k);
    }
    // Every word of one point from its stored form.
    __device__ __forceinline__ static void store_raw(T* __restrict__ f, size_t plane, size_t p, const Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 5; ++q) LBPS_ST(f + (size_t)(s * 5 + q) * plane + p, r.f[s][q]);
    }
    // The stored form store_point would write at p, in registers.
    __device__ __forceinline__ static void pack(size_t, const T (&x)[2][5], const KC<T>&, Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 5; ++q) r.f[s][q] = x[s][q];
    }
    // Equilibria of Eq. feq of both sets at lattice offset p for s[set] and
    // the lattice first moments (jx[set], jy[set]) (FP64 in), in stored form.
    // FP32 storage evaluates them in FP32 (from a and a_0 of the FP32
    // constants); FP64 storage in FP64.
    __device__ __forceinline__ static void eq_raw(size_t, const Consts& c, const double (&sv)[2],
                                                  const double (&jx)[2], const double (&jy)[2], const KC<T>& k,
                                                  Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if constexpr (sizeof(T) == 4) {
                const float sf = (float)sv[s], hx = mul_rn(0.5f, (float)jx[s]), hy = mul_rn(0.5f, (float)jy[s]);
                const float as = mul_rn(k.a[s], sf);
                r.f[s][0] = mul_rn(mul_rn(0.5f, k.two_a0[s]), sf);
                r.f[s][1] = add_rn(as, hx);
                r.f[s][2] = add_rn(as, hy);
                r.f[s][3] = sub_rn(as, hx);
                r.f[s][4] = sub_rn(as, hy);
            } else {
                const double as = c.a[s] * sv[s];
                r.f[s][0] = (T)(c.a0[s] * sv[s]);
                r.f[s][1] = (T)(as + 0.5 * jx[s]);
                r.f[s][2] = (T)(as + 0.5 * jy[s]);
                r.f[s][3] = (T)(as - 0.5 * jx[s]);
                r.f[s][4] = (T)(as - 0.5 * jy[s]);
            }
        }
    }
    // The same equilibria stored at p.
    __device__ __forceinline__ static void store_eq_point(T* __restrict__ f, size_t plane, size_t p, const Consts& c,
                                                          const double (&sv)[2], const double (&jx)[2],
                                                          const double (&jy)[2], const KC<T>& k) {
        Raw r;
        eq_raw(p, c, sv, jx, jy, k, r);
        store_raw(f, plane, p, r);
    }
    // One moving population alpha (1..4) of both sets.
    __device__ __forceinline__ static void store1_both(T* __restrict__ f, size_t plane, size_t p, int alpha,
                                                       const T (&v)[2], const KC<T>&) {
#pragma unroll
        for (int s = 0; s < 2; ++s) LBPS_ST(f + (size_t)(s * 5 + alpha) * plane + p, v[s]);
    }
    // The stored populations of set s, widened to FP64 (field output).
    __device__ __forceinline__ static void load5d(const T* __restrict__ f, size_t plane, size_t p, int s,
                                                  const KC<T>&, double (&x)[5]) {
#pragma unroll
        for (int q = 0; q < 5; ++q) x[q] = (double)LBPS_LD(f + (size_t)(s * 5 + q) * plane + p);
    }
};

// 16-bit value <-> its bits (the low or high half of a packed word)
template <typename H>
__device__ __forceinline__ float bits2f(unsigned b);
template <>
__device__ __forceinline__ float bits2f<__half>(unsigned b) { return __half2float(__ushort_as_half((unsigned short)b)); }
template <>
__device__ __forceinline__ float bits2f<__nv_bfloat16>(unsigned b) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)b));
}
template <typename H>
__device__ __forceinline__ unsigned f2bits(float v);
template <>
__device__ __forceinline__ unsigned f2bits<__half>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <>
__device__ __forceinline__ unsigned f2bits<__nv_bfloat16>(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Integer mixing function (the 32-bit finaliser of MurmurHash3): spreads
// every input bit over the output.
__device__ __forceinline__ unsigned mix32(unsigned h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// 16-bit code of v for the stored non-equilibrium sums: rounded to nearest,
// or (sr) stochastically, up with probability equal to the dropped fraction,
// the random bits a hash of the value and of `key` (the point and slot), so
// the result stays a deterministic function of the state.  When a_0 is near
// 1 the per-step changes of the sums lie near or below half a 16-bit ulp:
// rounding to nearest then makes nearly the same error every step and the
// errors add up, while unbiased rounding lets them average out.  With faster
// waves (a_0 further from 1) the errors of rounding to nearest decorrelate by
// themselves and stochastic rounding only adds variance.  The library rounds
// stochastically when a_{0,phi} >= 0.999 (KC::sr), for both formats.
template <typename H>
__device__ __forceinline__ unsigned f2bits_store(float v, unsigned key, bool sr);
template <>
__device__ __forceinline__ unsigned f2bits_store<__half>(float v, unsigned key, bool sr) {
    const float a = fabsf(v);
    // nearest for overflow and for subnormal halves (below 2^-14 more than
    // 13 bits are dropped)
    if (!sr || !(a < 65504.0f) || a < 6.103515625e-05f) return f2bits<__half>(v);
    const unsigned u = __float_as_uint(v);
    // 13 random bits added below the kept ones, then the magnitude truncated
    return __half_as_ushort(__float2half_rz(__uint_as_float(u + (mix32(u ^ mix32(key)) & 0x1fffu))));
}
template <>
__device__ __forceinline__ unsigned f2bits_store<__nv_bfloat16>(float v, unsigned key, bool sr) {
    if (!sr || !isfinite(v)) return f2bits<__nv_bfloat16>(v);
    const unsigned u = __float_as_uint(v);
    // adding below the kept bits rounds the magnitude up with the dropped
    // fraction's probability; a carry into the exponent is the next value up
    return (u + (mix32(u ^ mix32(key)) & 0xffffu)) >> 16;
}

// Populations of one set from f^0, J and the pair sums' deviations N
// (PopNeq16, PopBfp13): f^1 = r f^0 + (Nx + Jx) / 2, f^3 = r f^0 + (Nx - Jx) / 2
// and the same along y.
__device__ __forceinline__ void expand_pairs(float f0, float jx, float jy, float nx, float ny, float r,
                                             float (&x)[5]) {
    const float rf0 = mul_rn(r, f0);
    x[0] = f0;
    x[1] = fma_rn(0.5f, add_rn(nx, jx), rf0);
    x[3] = fma_rn(0.5f, sub_rn(nx, jx), rf0);
    x[2] = fma_rn(0.5f, add_rn(ny, jy), rf0);
    x[4] = fma_rn(0.5f, sub_rn(ny, jy), rf0);
}

template <typename H>
struct PopNeq16 {
    using V = float;
    using Base = float;
    static constexpr int kBytesPerPoint = 6 * 4 + 2 * 4;
    static constexpr bool kSplitStream = false;
    struct Raw {
        float m[2][3];   // f^0, Jx, Jy of each set
        unsigned w[2];   // packed Nx, Ny words (scaled)
    };
    __device__ __forceinline__ static const unsigned* words(const float* f, size_t plane) {
        return reinterpret_cast<const unsigned*>(f + 6 * plane);
    }
    __device__ __forceinline__ static unsigned* words(float* f, size_t plane) {
        return reinterpret_cast<unsigned*>(f + 6 * plane);
    }
    __device__ __forceinline__ static float half_of(unsigned w, int s, const KC<float>& k) {
        return mul_rn(bits2f<H>(s ? (w >> 16) : (w & 0xffffu)), k.inv_scale);
    }
    // key: the point's plane offset and the slot (set, pair) for the rounding
    __device__ __forceinline__ static unsigned enc_n(float pair_sum, float f0, float r, float scale,
                                                     unsigned key, bool sr) {
        return f2bits_store<H>(mul_rn(fma_rn(-2.0f * r, f0, pair_sum), scale), key, sr);
    }
    // Rounding key of slot (0..3: 2 set + pair) at plane offset p:
    // 4 (p + offset) + slot.  The empty asm keeps the compiler from folding
    // the offset into loop-invariant sums held in registers (which made the
    // 6-blocks-per-SM interior kernel spill); the offset stays a kernel
    // parameter read where it is added.
    __device__ __forceinline__ static unsigned key_of(size_t p, unsigned slot, const KC<float>& k) {
        unsigned x = (unsigned)p * 4u + slot;
        asm("" : "+r"(x));
        return x + k.key4;
    }
    __device__ __forceinline__ static void load_raw(const float* __restrict__ f, size_t plane, size_t p, bool ok,
                                                    Raw& r) {
        const unsigned* w = words(f, plane);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) r.m[s][q] = ok ? LBPS_LDG(f + (size_t)(s * 3 + q) * plane + p) : 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) r.w[q] = ok ? LBPS_LDG(w + (size_t)q * plane + p) : 0u;
    }
    __device__ __forceinline__ static void decode(const Raw& r, int s, const KC<float>& k, float (&x)[5]) {
        expand_pairs(r.m[s][0], r.m[s][1], r.m[s][2], half_of(r.w[0], s, k), half_of(r.w[1], s, k), k.r[s], x);
    }
    __device__ __forceinline__ static void load5(const float* __restrict__ f, size_t plane, size_t p, int s,
                                                 const KC<float>& k, float (&x)[5]) {
        const unsigned* w = words(f, plane);
        float m[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) m[q] = LBPS_LD(f + (size_t)(s * 3 + q) * plane + p);
        expand_pairs(m[0], m[1], m[2], half_of(LBPS_LD(w + p), s, k), half_of(LBPS_LD(w + plane + p), s, k), k.r[s], x);
    }
    // The same in FP64 (field output).
    __device__ __forceinline__ static void load5d(const float* __restrict__ f, size_t plane, size_t p, int s,
                                                  const KC<float>& k, double (&x)[5]) {
        const unsigned* w = words(f, plane);
        double f0 = LBPS_LD(f + (size_t)(s * 3) * plane + p);
        double jx = LBPS_LD(f + (size_t)(s * 3 + 1) * plane + p);
        double jy = LBPS_LD(f + (size_t)(s * 3 + 2) * plane + p);
        unsigned wx = LBPS_LD(w + p), wy = LBPS_LD(w + plane + p);
        double nx = (double)bits2f<H>(s ? (wx >> 16) : (wx & 0xffffu)) * (double)k.inv_scale;
        double ny = (double)bits2f<H>(s ? (wy >> 16) : (wy & 0xffffu)) * (double)k.inv_scale;
        double rf0 = (double)k.r[s] * f0;
        x[0] = f0;
        x[1] = rf0 + 0.5 * (nx + jx);
        x[3] = rf0 + 0.5 * (nx - jx);
        x[2] = rf0 + 0.5 * (ny + jy);
        x[4] = rf0 + 0.5 * (ny - jy);
    }
    __device__ __forceinline__ static void store_point(float* __restrict__ f, size_t plane, size_t p,
                                                       const float (&x)[2][5], const KC<float>& k) {
        unsigned wx = 0, wy = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            LBPS_ST(f + (size_t)(s * 3) * plane + p, x[s][0]);
            LBPS_ST(f + (size_t)(s * 3 + 1) * plane + p, sub_rn(x[s][1], x[s][3]));
            LBPS_ST(f + (size_t)(s * 3 + 2) * plane + p, sub_rn(x[s][2], x[s][4]));
            wx |= enc_n(add_rn(x[s][1], x[s][3]), x[s][0], k.r[s], k.scale, key_of(p, 2u * s, k),
                        k.sr)
                  << (16 * s);
            wy |= enc_n(add_rn(x[s][2], x[s][4]), x[s][0], k.r[s], k.scale,
                        key_of(p, 2u * s + 1u, k), k.sr)
                  << (16 * s);
        }
        unsigned* w = words(f, plane);
        LBPS_ST(w + p, wx);
        LBPS_ST(w + plane + p, wy);
    }
    // One moving population alpha (1..4) of both sets: the pair partner keeps
    // its value, so the pair's J and N are rewritten together.  Both sets'
    // N of a pair share one word, so the call owns that word; the library
    // rejects lattices 3 points wide along a non-periodic axis, the only shape
    // where two boundary sources stream into the same pair of one point.
    __device__ __forceinline__ static void store1_both(float* __restrict__ f, size_t plane, size_t p, int alpha,
                                                       const float (&v)[2], const KC<float>& k) {
        const int ax = (alpha == 1 || alpha == 3) ? 0 : 1;        // 0: x pair, 1: y pair
        const bool plus = alpha <= 2;                              // alpha = 1, 2: J = v - partner
        unsigned* wp = words(f, plane) + (size_t)ax * plane + p;
        const unsigned w = LBPS_LD(wp);
        unsigned out = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            float* jp = f + (size_t)(s * 3 + 1 + ax) * plane + p;
            const float f0 = LBPS_LD(f + (size_t)(s * 3) * plane + p);
            const float j = LBPS_LD(jp);
            const float nn = half_of(w, s, k);
            const float rf0 = mul_rn(k.r[s], f0);
            const float partner = plus ? fma_rn(0.5f, sub_rn(nn, j), rf0) : fma_rn(0.5f, add_rn(nn, j), rf0);
            LBPS_ST(jp, plus ? sub_rn(v[s], partner) : sub_rn(partner, v[s]));
            out |= enc_n(add_rn(v[s], partner), f0, k.r[s], k.scale,
                         key_of(p, 2u * s + (unsigned)ax, k), k.sr)
                   << (16 * s);
        }
        LBPS_ST(wp, out);
    }
    // The stored form store_point would write at p, in registers.
    __device__ __forceinline__ static void pack(size_t p, const float (&x)[2][5], const KC<float>& k, Raw& r) {
        unsigned wx = 0, wy = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            r.m[s][0] = x[s][0];
            r.m[s][1] = sub_rn(x[s][1], x[s][3]);
            r.m[s][2] = sub_rn(x[s][2], x[s][4]);
            wx |= enc_n(add_rn(x[s][1], x[s][3]), x[s][0], k.r[s], k.scale, key_of(p, 2u * s, k), k.sr)
                  << (16 * s);
            wy |= enc_n(add_rn(x[s][2], x[s][4]), x[s][0], k.r[s], k.scale, key_of(p, 2u * s + 1u, k), k.sr)
                  << (16 * s);
        }
        r.w[0] = wx;
        r.w[1] = wy;
    }
    // Every word of one point from its stored form.
    __device__ __forceinline__ static void store_raw(float* __restrict__ f, size_t plane, size_t p, const Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) LBPS_ST(f + (size_t)(s * 3 + q) * plane + p, r.m[s][q]);
        unsigned* w = words(f, plane);
        LBPS_ST(w + p, r.w[0]);
        LBPS_ST(w + plane + p, r.w[1]);
    }
    // Equilibria of Eq. feq of both sets at lattice offset p (the rounding key),
    // in FP32 and in stored form: J = (jx, jy) and the pair sums' deviation
    // 2 a s - 2 r f^0 from the stored f^0 (zero up to rounding), scaled.
    __device__ __forceinline__ static void eq_raw(size_t p, const Consts&, const double (&sv)[2],
                                                  const double (&jx)[2], const double (&jy)[2],
                                                  const KC<float>& k, Raw& r) {
        unsigned w = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float sf = (float)sv[s];
            const float f0 = mul_rn(mul_rn(0.5f, k.two_a0[s]), sf);
            r.m[s][0] = f0;
            r.m[s][1] = (float)jx[s];
            r.m[s][2] = (float)jy[s];
            const float dev = mul_rn(fma_rn(-2.0f * k.r[s], f0, mul_rn(k.two_a[s], sf)), k.scale);
            w |= f2bits_store<H>(dev, key_of(p, 2u * s, k), k.sr) << (16 * s);
        }
        r.w[0] = w;
        r.w[1] = w;
    }
    // The same equilibria stored at p, each packed word written once.
    __device__ __forceinline__ static void store_eq_point(float* __restrict__ f, size_t plane, size_t p,
                                                          const Consts& c, const double (&sv)[2],
                                                          const double (&jx)[2], const double (&jy)[2],
                                                          const KC<float>& k) {
        Raw r;
        eq_raw(p, c, sv, jx, jy, k, r);
        store_raw(f, plane, p, r);
    }
};

// ---- BFP13: block floating point, two values per 32-bit word
//
// Both values of a word share a 4-bit exponent E; each has a sign and a
// 13-bit magnitude m (no hidden bit), value = m 2^(E-13):
//   bits 31..28 E, bit 27 sign of a, 26..14 m of a, bit 13 sign of b,
//   12..0 m of b.
// E is the smallest exponent at which the larger magnitude rounds to at most
// 8191, so the larger value keeps 13 significant bits (IEEE half has 11) and
// the smaller one the same absolute step; the range is m 2^-13 .. 32761.99.
// E = 15 with m = 8191 is infinity (overflow; non-finite input).  Rounding
// is to nearest, ties to even.
__device__ __forceinline__ void bfp13_decode(unsigned w, float& a, float& b) {
    // FP32 2^E (1 + m 2^-13) less 2^E: m 2^(E-13), exactly; the magnitudes
    // moved into the top of the FP32 fraction field
    const unsigned eb = ((w >> 28) + 127u) << 23;
    const float base = __uint_as_float(eb);
    float xa = __uint_as_float(eb | ((w >> 4) & 0x7ffc00u)) - base;
    float xb = __uint_as_float(eb | ((w << 10) & 0x7ffc00u)) - base;
    if ((w & 0xf7ffc000u) == 0xf7ffc000u) xa = __uint_as_float(0x7f800000u);
    if ((w & 0xf0001fffu) == 0xf0001fffu) xb = __uint_as_float(0x7f800000u);
    a = __uint_as_float(__float_as_uint(xa) | ((w << 4) & 0x80000000u));
    b = __uint_as_float(__float_as_uint(xb) | ((w << 18) & 0x80000000u));
}
__device__ __forceinline__ unsigned bfp13_encode(float a, float b) {
    const unsigned sa = __float_as_uint(a) >> 31, sb = __float_as_uint(b) >> 31;
    const float xa = fabsf(a), xb = fabsf(b);
    const unsigned signs = (sa << 27) | (sb << 13);
    // overflow (and NaN): both values infinite
    if (!(xa < 32762.0f) || !(xb < 32762.0f)) return 0xf7ffdfffu | signs;
    // E = floor(log2 big) + 1 from the FP32 exponent field, at least 0 (zero,
    // subnormals), and one more where big 2^(13-E) would round to 2^13: where
    // the fraction field is at least 2^23 - 2^10, which adding 2^10 to the
    // bits carries into the exponent field
    const int E = max((int)((__float_as_uint(fmaxf(xa, xb)) + 0x400u) >> 23) - 126, 0);
    const float sc = __uint_as_float((unsigned)(140 - E) << 23);   // 2^(13-E)
    const unsigned ma = __float2uint_rn(xa * sc), mb = __float2uint_rn(xb * sc);
    return ((unsigned)E << 28) | signs | (ma << 14) | mb;
}

// PopBfp13: per set f^0, Jx, Jy in FP32 as in PopNeq16, and the set's two
// non-equilibrium pair sums Nx, Ny times 2^e in one BFP13 word (a = Nx,
// b = Ny): plane 6 holds phi's word, plane 7 psi's; 32 bytes per point, as
// PopNeq16, with 13-bit magnitudes instead of 11 significant bits.  Always
// rounded to nearest (KC::sr is not used).  Writing one streamed pair of a
// point rewrites the word of each set, which also holds the other pair, so
// the boundary reset writes its x and its y streams in two passes
// (kSplitStream); re-encoding the other pair is exact unless the new value
// raises the shared exponent.
struct PopBfp13 {
    using V = float;
    using Base = float;
    static constexpr int kBytesPerPoint = 6 * 4 + 2 * 4;
    static constexpr bool kSplitStream = true;
    struct Raw {
        float m[2][3];   // f^0, Jx, Jy of each set
        unsigned w[2];   // the BFP13 word (Nx, Ny scaled) of each set
    };
    __device__ __forceinline__ static const unsigned* words(const float* f, size_t plane) {
        return reinterpret_cast<const unsigned*>(f + 6 * plane);
    }
    __device__ __forceinline__ static unsigned* words(float* f, size_t plane) {
        return reinterpret_cast<unsigned*>(f + 6 * plane);
    }
    // Nx, Ny of one set from its word
    __device__ __forceinline__ static void n_of(unsigned w, const KC<float>& k, float& nx, float& ny) {
        bfp13_decode(w, nx, ny);
        nx = mul_rn(nx, k.inv_scale);
        ny = mul_rn(ny, k.inv_scale);
    }
    // the scaled deviation of a pair sum from 2 r f^0
    __device__ __forceinline__ static float scaled_n(float pair_sum, float f0, float r, float scale) {
        return mul_rn(fma_rn(-2.0f * r, f0, pair_sum), scale);
    }
    __device__ __forceinline__ static unsigned enc_set(const float (&x)[5], float r, float scale) {
        return bfp13_encode(scaled_n(add_rn(x[1], x[3]), x[0], r, scale), scaled_n(add_rn(x[2], x[4]), x[0], r, scale));
    }
    __device__ __forceinline__ static void load_raw(const float* __restrict__ f, size_t plane, size_t p, bool ok,
                                                    Raw& r) {
        const unsigned* w = words(f, plane);
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) r.m[s][q] = ok ? LBPS_LDG(f + (size_t)(s * 3 + q) * plane + p) : 0.0f;
#pragma unroll
        for (int q = 0; q < 2; ++q) r.w[q] = ok ? LBPS_LDG(w + (size_t)q * plane + p) : 0u;
    }
    __device__ __forceinline__ static void decode(const Raw& r, int s, const KC<float>& k, float (&x)[5]) {
        float nx, ny;
        n_of(r.w[s], k, nx, ny);
        expand_pairs(r.m[s][0], r.m[s][1], r.m[s][2], nx, ny, k.r[s], x);
    }
    __device__ __forceinline__ static void load5(const float* __restrict__ f, size_t plane, size_t p, int s,
                                                 const KC<float>& k, float (&x)[5]) {
        float m[3], nx, ny;
#pragma unroll
        for (int q = 0; q < 3; ++q) m[q] = LBPS_LD(f + (size_t)(s * 3 + q) * plane + p);
        n_of(LBPS_LD(words(f, plane) + (size_t)s * plane + p), k, nx, ny);
        expand_pairs(m[0], m[1], m[2], nx, ny, k.r[s], x);
    }
    // The same in FP64 (field output).
    __device__ __forceinline__ static void load5d(const float* __restrict__ f, size_t plane, size_t p, int s,
                                                  const KC<float>& k, double (&x)[5]) {
        double f0 = LBPS_LD(f + (size_t)(s * 3) * plane + p);
        double jx = LBPS_LD(f + (size_t)(s * 3 + 1) * plane + p);
        double jy = LBPS_LD(f + (size_t)(s * 3 + 2) * plane + p);
        float ax, ay;
        bfp13_decode(LBPS_LD(words(f, plane) + (size_t)s * plane + p), ax, ay);
        double nx = (double)ax * (double)k.inv_scale, ny = (double)ay * (double)k.inv_scale;
        double rf0 = (double)k.r[s] * f0;
        x[0] = f0;
        x[1] = rf0 + 0.5 * (nx + jx);
        x[3] = rf0 + 0.5 * (nx - jx);
        x[2] = rf0 + 0.5 * (ny + jy);
        x[4] = rf0 + 0.5 * (ny - jy);
    }
    __device__ __forceinline__ static void store_point(float* __restrict__ f, size_t plane, size_t p,
                                                       const float (&x)[2][5], const KC<float>& k) {
        unsigned* w = words(f, plane);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            LBPS_ST(f + (size_t)(s * 3) * plane + p, x[s][0]);
            LBPS_ST(f + (size_t)(s * 3 + 1) * plane + p, sub_rn(x[s][1], x[s][3]));
            LBPS_ST(f + (size_t)(s * 3 + 2) * plane + p, sub_rn(x[s][2], x[s][4]));
            LBPS_ST(w + (size_t)s * plane + p, enc_set(x[s], k.r[s], k.scale));
        }
    }
    // store_point for an interior point whose moving populations flagged in
    // prov (1: f^1, 2: f^3, 4: f^2, 8: f^4) streamed in from boundary points:
    // the reset overwrites each of them and keeps only its pair partner
    // (store1_both).  Such a pair is stored as N = 0 and the J that gives the
    // partner back, J = 2 (r f^0 - f^3) or 2 (f^1 - r f^0), so that the
    // provisional value neither sets the word's exponent (and costs the other
    // pair its precision) nor passes through the 13-bit rounding.
    __device__ __forceinline__ static void store_point_pins(float* __restrict__ f, size_t plane, size_t p,
                                                            const float (&x)[2][5], const KC<float>& k, int prov) {
        unsigned* w = words(f, plane);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float f0 = x[s][0], rf0 = mul_rn(k.r[s], f0);
            float jx = sub_rn(x[s][1], x[s][3]), jy = sub_rn(x[s][2], x[s][4]);
            float nx = scaled_n(add_rn(x[s][1], x[s][3]), f0, k.r[s], k.scale);
            float ny = scaled_n(add_rn(x[s][2], x[s][4]), f0, k.r[s], k.scale);
            if (prov & 3) {
                jx = mul_rn(2.0f, (prov & 1) ? sub_rn(rf0, x[s][3]) : sub_rn(x[s][1], rf0));
                nx = 0.0f;
            }
            if (prov & 12) {
                jy = mul_rn(2.0f, (prov & 4) ? sub_rn(rf0, x[s][4]) : sub_rn(x[s][2], rf0));
                ny = 0.0f;
            }
            LBPS_ST(f + (size_t)(s * 3) * plane + p, f0);
            LBPS_ST(f + (size_t)(s * 3 + 1) * plane + p, jx);
            LBPS_ST(f + (size_t)(s * 3 + 2) * plane + p, jy);
            LBPS_ST(w + (size_t)s * plane + p, bfp13_encode(nx, ny));
        }
    }
    // One moving population alpha (1..4) of both sets: the pair partner keeps
    // its value, so the pair's J and N are rewritten together, and each set's
    // word with the N of the other pair (decoded and encoded again).  The
    // call owns both words of the point: the reset writes x streams and y
    // streams in separate passes, and the library rejects lattices 3 points
    // wide along a non-periodic axis (two sources into one pair).
    __device__ __forceinline__ static void store1_both(float* __restrict__ f, size_t plane, size_t p, int alpha,
                                                       const float (&v)[2], const KC<float>& k) {
        const int ax = (alpha == 1 || alpha == 3) ? 0 : 1;        // 0: x pair, 1: y pair
        const bool plus = alpha <= 2;                              // alpha = 1, 2: J = v - partner
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            unsigned* wp = words(f, plane) + (size_t)s * plane + p;
            float n[2];
            bfp13_decode(LBPS_LD(wp), n[0], n[1]);
            float* jp = f + (size_t)(s * 3 + 1 + ax) * plane + p;
            const float f0 = LBPS_LD(f + (size_t)(s * 3) * plane + p);
            const float j = LBPS_LD(jp);
            const float nn = mul_rn(ax ? n[1] : n[0], k.inv_scale);
            const float rf0 = mul_rn(k.r[s], f0);
            const float partner = plus ? fma_rn(0.5f, sub_rn(nn, j), rf0) : fma_rn(0.5f, add_rn(nn, j), rf0);
            LBPS_ST(jp, plus ? sub_rn(v[s], partner) : sub_rn(partner, v[s]));
            const float nv = scaled_n(add_rn(v[s], partner), f0, k.r[s], k.scale);
            LBPS_ST(wp, ax ? bfp13_encode(n[0], nv) : bfp13_encode(nv, n[1]));
        }
    }
    // The stored form store_point would write at p, in registers.
    __device__ __forceinline__ static void pack(size_t, const float (&x)[2][5], const KC<float>& k, Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            r.m[s][0] = x[s][0];
            r.m[s][1] = sub_rn(x[s][1], x[s][3]);
            r.m[s][2] = sub_rn(x[s][2], x[s][4]);
            r.w[s] = enc_set(x[s], k.r[s], k.scale);
        }
    }
    // Every word of one point from its stored form.
    __device__ __forceinline__ static void store_raw(float* __restrict__ f, size_t plane, size_t p, const Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int q = 0; q < 3; ++q) LBPS_ST(f + (size_t)(s * 3 + q) * plane + p, r.m[s][q]);
        unsigned* w = words(f, plane);
        LBPS_ST(w + p, r.w[0]);
        LBPS_ST(w + plane + p, r.w[1]);
    }
    // Equilibria of Eq. feq of both sets, in FP32 and in stored form (as
    // PopNeq16::eq_raw; p unused, no rounding keys).
    __device__ __forceinline__ static void eq_raw(size_t, const Consts&, const double (&sv)[2],
                                                  const double (&jx)[2], const double (&jy)[2],
                                                  const KC<float>& k, Raw& r) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float sf = (float)sv[s];
            const float f0 = mul_rn(mul_rn(0.5f, k.two_a0[s]), sf);
            r.m[s][0] = f0;
            r.m[s][1] = (float)jx[s];
            r.m[s][2] = (float)jy[s];
            const float dev = mul_rn(fma_rn(-2.0f * k.r[s], f0, mul_rn(k.two_a[s], sf)), k.scale);
            r.w[s] = bfp13_encode(dev, dev);
        }
    }
    __device__ __forceinline__ static void store_eq_point(float* __restrict__ f, size_t plane, size_t p,
                                                          const Consts& c, const double (&sv)[2],
                                                          const double (&jx)[2], const double (&jy)[2],
                                                          const KC<float>& k) {
        Raw r;
        eq_raw(p, c, sv, jx, jy, k, r);
        store_raw(f, plane, p, r);
    }
};

}  // namespace lbps
