// C ABI of the plane-strain LBM library (declarations and contracts in
// include/lbps.h).  Host-side work only: validation, the rectangle helper,
// the device memory layout, and enqueueing the kernels of lbps_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lbps.h"
#include "lbps_launch.h"
#include "lbps_state.h"

using lbps::BNode;
using lbps::Consts;
using lbps::Geo;
using lbps::KC;
using lbps::Layout;
using lbps::View;

namespace {

constexpr size_t kAlign = 256;
// a_{0,phi} from which 16-bit storage rounds stochastically: at 0.9999 it cut
// the error of FP16 on 10^4-step waves 5x; at 0.99 and below rounding to
// nearest was 1.4x better
constexpr double kStochasticA0 = 0.999;
constexpr size_t kStagingMax = size_t(8) << 20;  // host read/write staging, bytes

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool finite_positive(double x) { return std::isfinite(x) && x > 0.0; }

int validate_params(const lbps_params* p) {
    if (!p) return LBPS_ERR_INVALID;
    if (p->nx < 3 || p->ny < 3 || p->nx > (1 << 24) || p->ny > (1 << 24)) return LBPS_ERR_INVALID;
    if (!finite_positive(p->mu) || !finite_positive(p->rho) || !std::isfinite(p->lambda)) return LBPS_ERR_INVALID;
    if (!(p->lambda + 2.0 * p->mu > 0.0) || !finite_positive(p->dh)) return LBPS_ERR_INVALID;
    if (!(p->a0_phi >= 0.0 && p->a0_phi < 1.0)) return LBPS_ERR_INVALID;
    if (p->bc_feq_mode != 0 && p->bc_feq_mode != 1) return LBPS_ERR_INVALID;
    if (p->bc_j_mode != 0 && p->bc_j_mode != 1) return LBPS_ERR_INVALID;
    if (p->sync_every < 0) return LBPS_ERR_INVALID;
    if (p->storage < LBPS_STORAGE_F32 || p->storage > LBPS_STORAGE_BFP13) return LBPS_ERR_INVALID;
    if (p->pop_scale_exp < -100 || p->pop_scale_exp > 100) return LBPS_ERR_INVALID;
    if ((p->periodic_x != 0 && p->periodic_x != 1) || (p->periodic_y != 0 && p->periodic_y != 1))
        return LBPS_ERR_INVALID;
    // 16-bit storage rewrites a population pair as a whole; on a lattice 3 points
    // wide along a non-periodic axis two boundary sources stream into the same
    // pair of one point, which that cannot express.
    if (lbps::storage_is16(p->storage) &&
        ((!p->periodic_x && p->nx == 3) || (!p->periodic_y && p->ny == 3)))
        return LBPS_ERR_INVALID;
    return LBPS_OK;
}

// general: node types from a type plane (void points, given cells); nb_general:
// the number of boundary points then (a rectangle's is its perimeter).
Layout make_layout(const lbps_params* p, bool general = false, int nb_general = 0) {
    Layout L{};
    L.g.nx = p->nx;
    L.g.ny = p->ny;
    L.g.px = (p->nx + 31) / 32 * 32;
    L.g.periodic_x = p->periodic_x;
    L.g.periodic_y = p->periodic_y;
    L.g.general = general ? 1 : 0;
    L.g.plane = (size_t)L.g.px * (size_t)p->ny;
    const size_t per_point =
        lbps::with_policy(p->storage, [](auto pol) { return (size_t)decltype(pol)::kBytesPerPoint; });
    L.f_bytes = align_up(L.g.plane * per_point);
    L.u_bytes = align_up(4 * L.g.plane * 8);
    L.nb = general ? nb_general : lbps::perim_count(L.g);
    L.g.mplane = ((size_t)L.nb + 31) / 32 * 32;
    L.m_bytes = align_up(L.g.mplane * per_point);
    L.s_bytes = align_up((general ? 5 : 2) * (size_t)L.nb * 3 * sizeof(double));
    L.copy_bytes = L.f_bytes + L.u_bytes + L.m_bytes + L.s_bytes;
    size_t off = 0;
    L.off_copy[0] = off;
    off += L.copy_bytes;
    L.off_copy[1] = off;
    off += L.copy_bytes;
    L.off_bn = off;
    off += align_up((size_t)L.nb * sizeof(BNode));
    L.off_type = off;
    if (general) off += align_up(L.g.plane);
    L.off_gap = off;  // general: 2 ints per strip of the interior kernel
    if (general)
        off += align_up((size_t)2 * (size_t)((p->nx + lbps::kBatchStripCols - 1) / lbps::kBatchStripCols) * sizeof(int));
    L.off_part = off;
    off += align_up((size_t)lbps::kNormBlocks * 4 * sizeof(double));
    L.off_out = off;
    off += kAlign;
    L.off_flag = off;
    off += kAlign;
    size_t dense = 5 * (size_t)p->nx * (size_t)p->ny * sizeof(double);
    L.staging_bytes = align_up(dense < kStagingMax ? dense : kStagingMax);
    L.off_staging = off;
    off += L.staging_bytes;
    L.total = off;
    return L;
}

template <typename T>
KC<T> make_kc(double a_phi, double a_psi, double cd2, double cs2, double dh) {
    KC<T> k;
    double a[2] = {a_phi, a_psi};
    for (int s = 0; s < 2; ++s) {
        T at = (T)a[s];
        T a0t = (T)(1.0 - 4.0 * (double)at);
        k.a[s] = at;
        k.two_a[s] = (T)2 * at;
        k.eight_a[s] = (T)8 * at;
        k.two_a0[s] = (T)2 * a0t;
    }
    k.cd2h = (T)(cd2 * 0.5 / dh);
    k.cs2h = (T)(cs2 * 0.5 / dh);
    for (int s = 0; s < 2; ++s) k.r[s] = (T)(a[s] / (1.0 - 4.0 * a[s]));
    k.scale = (T)1;
    k.sr = 0;
    k.inv_scale = (T)1;
    k.key4 = 0;
    return k;
}

// The boundary list of a lattice, checked against the node types.
struct Boundary {
    bool general = false;
    std::vector<BNode> bn;
};

// Rectangle (no void points, no cells): the outer ring in perimeter order,
// cells by reading R6 (computed in the kernel from the indices).  General
// geometry (reading R14): every body point with a neighbour outside the body,
// in row-major order, with its cell (given, or the clipped square of R6),
// its body and interior neighbours; every body point must have a difference
// stencil along both axes.
int build_boundary(const lbps_params* p, const uint8_t* node_type, const double* bc_value, const double* cell,
                   Boundary& out) {
    const int nx = p->nx, ny = p->ny;
    bool any_void = false;
    if (node_type)
        for (size_t k = 0; k < (size_t)nx * ny; ++k) {
            if (node_type[k] > 3) return LBPS_ERR_INVALID;
            any_void = any_void || node_type[k] == 3;
        }
    out.general = any_void || cell != nullptr;
    out.bn.clear();
    const int DX[4] = {1, 0, -1, 0};
    const int DY[4] = {0, 1, 0, -1};
    auto type_at = [&](int i, int j) { return node_type ? node_type[(size_t)j * nx + i] : (uint8_t)LBPS_INTERIOR; };
    auto body = [&](int i, int j) {
        if (i < 0 || i >= nx) {
            if (!p->periodic_x) return false;
            i = (i + nx) % nx;
        }
        if (j < 0 || j >= ny) {
            if (!p->periodic_y) return false;
            j = (j + ny) % ny;
        }
        return type_at(i, j) != 3;
    };
    auto boundary = [&](int i, int j) {
        if (!body(i, j)) return false;
        for (int d = 0; d < 4; ++d)
            if (!body(i + DX[d], j + DY[d])) return true;
        return false;
    };
    auto bvalue = [&](size_t k, double& bx, double& by) {
        bx = bc_value ? bc_value[2 * k] : 0.0;
        by = bc_value ? bc_value[2 * k + 1] : 0.0;
        return std::isfinite(bx) && std::isfinite(by);
    };
    if (!out.general) {
        Geo g{};
        g.nx = nx;
        g.ny = ny;
        g.periodic_x = p->periodic_x;
        g.periodic_y = p->periodic_y;
        const int nb = lbps::perim_count(g);
        out.bn.assign((size_t)nb, BNode{});
        std::vector<char> seen((size_t)nb, 0);
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                size_t k = (size_t)j * nx + i;
                int t = type_at(i, j);
                if (!lbps::is_boundary(i, j, g)) {
                    if (t != LBPS_INTERIOR) return LBPS_ERR_INVALID;
                    continue;
                }
                if (t != LBPS_NEUMANN && t != LBPS_DIRICHLET) return LBPS_ERR_INVALID;
                double bx, by;
                if (!bvalue(k, bx, by)) return LBPS_ERR_INVALID;
                int q = lbps::perim_index(i, j, g);
                if (q < 0 || q >= nb || seen[q]) return LBPS_ERR_INVALID;
                seen[q] = 1;
                // the one interior neighbour of an edge point (none at corners)
                bool l = !p->periodic_x && i == 0, r = !p->periodic_x && i == nx - 1;
                bool b = !p->periodic_y && j == 0, tp = !p->periodic_y && j == ny - 1;
                int smask = ((l || r) && (b || tp)) ? 0 : l ? 1 : r ? 4 : b ? 2 : 8;
                BNode node{};
                node.i = i;
                node.j = j;
                node.type = t;
                node.smask = smask;
                node.bx = bx;
                node.by = by;
                out.bn[q] = node;
            }
        }
        return LBPS_OK;
    }
    const double half = 0.5 * p->dh;
    const bool pairs16 = lbps::storage_is16(p->storage);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            int t = type_at(i, j);
            if (t == 3) continue;
            for (int ax = 0; ax < 2; ++ax) {  // a difference stencil along x and y
                int dx = ax == 0, dy = ax == 1;
                bool hp = body(i + dx, j + dy), hm = body(i - dx, j - dy);
                bool ok = (hp && hm) || (hp && body(i + 2 * dx, j + 2 * dy)) || (hm && body(i - 2 * dx, j - 2 * dy));
                if (!ok) return LBPS_ERR_INVALID;
            }
            const bool bnd = boundary(i, j);
            if (!bnd) {
                if (t != LBPS_INTERIOR) return LBPS_ERR_INVALID;
                // 16-bit storage writes a population pair as a whole: no point
                // may receive one pair from boundary sources on both sides
                if (pairs16 && ((boundary(i - 1, j) && boundary(i + 1, j)) || (boundary(i, j - 1) && boundary(i, j + 1))))
                    return LBPS_ERR_INVALID;
                continue;
            }
            if (t != LBPS_NEUMANN && t != LBPS_DIRICHLET) return LBPS_ERR_INVALID;
            BNode node{};
            node.i = i;
            node.j = j;
            node.type = t;
            if (!bvalue(k, node.bx, node.by)) return LBPS_ERR_INVALID;
            bool has[4];
            for (int d = 0; d < 4; ++d) {
                has[d] = body(i + DX[d], j + DY[d]);
                if (has[d]) node.nbmask |= 1 << d;
                if (has[d] && !boundary(i + DX[d], j + DY[d])) node.smask |= 1 << d;
            }
            if (t == LBPS_NEUMANN) {
                double vol;
                if (cell) {
                    vol = cell[5 * k];
                    for (int d = 0; d < 4; ++d) node.l[d] = cell[5 * k + 1 + d];
                    bool ok = std::isfinite(vol) && vol > 0.0;
                    for (int d = 0; d < 4; ++d) ok = ok && std::isfinite(node.l[d]) && node.l[d] >= 0.0;
                    if (!ok) return LBPS_ERR_INVALID;
                } else {  // reading R6: the square of side dh clipped at missing neighbours
                    double wx = (has[2] ? half : 0.0) + (has[0] ? half : 0.0);
                    double wy = (has[3] ? half : 0.0) + (has[1] ? half : 0.0);
                    vol = wx * wy;
                    node.l[0] = has[0] ? wy : 0.0;
                    node.l[1] = has[1] ? wx : 0.0;
                    node.l[2] = has[2] ? wy : 0.0;
                    node.l[3] = has[3] ? wx : 0.0;
                    if (!(vol > 0.0)) return LBPS_ERR_INVALID;
                }
                node.inv_m = 1.0 / (p->rho * vol);
            }
            out.bn.push_back(node);
        }
    }
    return LBPS_OK;
}

// 64-bit FNV-1a over bytes, for the set-up fingerprint of saved states.
struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t q = 0; q < n; ++q) {
            h ^= b[q];
            h *= 1099511628211ull;
        }
    }
    template <typename T>
    void add(const T& v) {
        add(&v, sizeof(T));
    }
};

// Fingerprint of what a state's meaning depends on besides its own bytes:
// the parameters of the method and the boundary description (boundary list
// with its values and cells; for a general geometry also the node types).
uint64_t setup_hash(const lbps_params* p, const Boundary& bd, const uint8_t* node_type) {
    Fnv f;
    f.add(p->nx);
    f.add(p->ny);
    f.add(p->lambda);
    f.add(p->mu);
    f.add(p->rho);
    f.add(p->dh);
    f.add(p->a0_phi);
    f.add(p->periodic_x);
    f.add(p->periodic_y);
    f.add(p->bc_feq_mode);
    f.add(p->bc_j_mode);
    f.add(p->sync_every);
    f.add(p->storage);
    for (const BNode& q : bd.bn) {
        f.add(q.i);
        f.add(q.j);
        f.add(q.type);
        f.add(q.smask);
        f.add(q.bx);
        f.add(q.by);
        f.add(q.inv_m);
        f.add(q.l);
        f.add(q.nbmask);
    }
    if (bd.general && node_type) f.add(node_type, (size_t)p->nx * (size_t)p->ny);
    return f.h;
}

}  // namespace

namespace {

int cuda_ok(cudaError_t e) { return e == cudaSuccess ? LBPS_OK : LBPS_ERR_CUDA; }

// Next free event of the profiling pool (created on demand).
cudaEvent_t next_event(lbps_lattice* lat) {
    if (lat->ev_used == lat->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        lat->ev_pool.push_back(e);
    }
    return lat->ev_pool[lat->ev_used++];
}

// Records an event on a stream (default: the lattice's) when profiling; the
// pair (start, end) of a kernel is two consecutive pool entries.
cudaError_t prof_mark(lbps_lattice* lat, cudaStream_t st = nullptr) {
    if (!lat->prof) return cudaSuccess;
    cudaEvent_t e = next_event(lat);
    if (!e) return cudaErrorMemoryAllocation;
    return cudaEventRecord(e, st ? st : lat->st);
}

// Boundary passes [pass_lo, pass_hi) of one step (1 Newmark, 2 reset; 0, the
// stresses of copy a, only after the initialisation), on stream st (default:
// the lattice's).  timed = false leaves them out of lbps_profile (a pass
// beside the interior kernel waits for free SMs, so events around it would
// not measure it).
cudaError_t boundary_passes(lbps_lattice* lat, int a, int b, int pass_lo, int pass_hi,
                            cudaStream_t st = nullptr, bool timed = true) {
    if (lat->L.nb == 0) return cudaSuccess;
    if (!st) st = lat->st;
    const bool prof = lat->prof;
    lat->prof = prof && timed;
    cudaError_t e = prof_mark(lat, st);
    if (e == cudaSuccess)
        e = lbps::with_policy(lat->p.storage, [&](auto pol) {
            using P = decltype(pol);
            return lbps::launch_boundary<P>(lat->L.g, lat->c, lat->kc<P>(), lat->view<P>(a), lat->view<P>(b),
                                            lat->bn(), lat->L.nb, lat->flag(), lat->tstep(), st, pass_lo,
                                            pass_hi);
        });
    if (e == cudaSuccess) e = prof_mark(lat, st);
    if (e == cudaSuccess && lat->prof) lat->ev_kind.push_back(1);
    lat->prof = prof;
    return e;
}

// One time step: the boundary Newmark pass, the interior kernel, then the
// boundary reset (which reads the interior kernel's new u, overwrites the
// populations streamed from boundary points and leaves the stresses of the
// new u for the next step).  The Newmark pass runs on the side stream beside
// the interior kernel: it reads copy A and writes only the boundary points'
// u, du/dt of copy B, which the interior kernel does not touch; the reset
// waits for both.
int run_step(lbps_lattice* lat) {
    int a = lat->cur, b = lat->cur ^ 1;
    const bool overlap = lat->side && lat->L.nb > 0;
    cudaError_t e = cudaSuccess;
    if (overlap) {
        e = cudaEventRecord(lat->fork, lat->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->side, lat->fork, 0);
        if (e == cudaSuccess) e = boundary_passes(lat, a, b, 1, 2, lat->side, false);
        if (e == cudaSuccess) e = cudaEventRecord(lat->join, lat->side);
    } else {
        e = boundary_passes(lat, a, b, 1, 2);
    }
    if (e == cudaSuccess) e = prof_mark(lat);
    if (e == cudaSuccess)
        e = lbps::with_policy(lat->p.storage, [&](auto pol) {
            using P = decltype(pol);
            return lbps::launch_bulk<P>(lat->L.g, lat->c, lat->kc<P>(), lat->view<P>(a), lat->view<P>(b),
                                        lat->flag(), lat->st, lat->tuning);
        });
    if (e == cudaSuccess) e = prof_mark(lat);
    if (e == cudaSuccess && lat->prof) lat->ev_kind.push_back(0);
    if (e == cudaSuccess && overlap) e = cudaStreamWaitEvent(lat->st, lat->join, 0);
    if (e == cudaSuccess) e = boundary_passes(lat, a, b, 2, 3);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    lat->cur = b;
    lat->steps += 1;
    return LBPS_OK;
}

// Two steps per sweep apply to rectangles without periodic axes, at least
// 16 points a side, with the scratch copy allocated and per-kernel timing off.
bool pair_ok(const lbps_lattice* lat) {
    const lbps::Geo& g = lat->L.g;
    return lat->xmem && lat->side && !g.general && !g.periodic_x && !g.periodic_y && g.nx >= 16 && g.ny >= 16 &&
           lat->L.nb > 0;
}

// Below this many points a lattice takes its pairs of steps as a batch of
// itself (lbps_batch_set_step_pairs): four launches a pair, the two-step
// strips and the first step's frame strips in one persistent kernel, where
// run_pair's concurrent chain on the second stream costs thirteen launches.
// Measured (FP32 pulses, CUDA graphs, run_pair's second stream at the
// greatest priority): 2048^2 46.3 against 37.9 GLUPS, 3072^2 56.8 against
// 56.9; from 4096^2 run_pair is faster (68.8 against 63.0).
constexpr int64_t kSoloPairsMaxPoints = 12ll << 20;

bool solo_pairs(const lbps_lattice* lat) {
    return pair_ok(lat) && !lat->prof && lat->p.sync_every == 0 &&
           (int64_t)lat->L.g.nx * (int64_t)lat->L.g.ny < kSoloPairsMaxPoints;
}

void drop_solo(lbps_lattice* lat) {
    if (lat->solo) lbps_batch_destroy(lat->solo);
    lat->solo = nullptr;
}

// Steps n and n + 1 in one sweep of the interior.  Copy A (current) holds
// step n, copy B receives step n + 2, the scratch copy X step n + 1 where the
// boundary rules need it:
//   side stream: Newmark(n) A -> X; the interior kernel on the points 1..3
//   from the edges, A -> X; reset(n) A, X -> X; Newmark(n + 1) X -> B; the
//   interior kernel on the points 1..2 from the edges, X -> B; reset(n + 1)
//   X, B -> B (the order of two single steps, on X and B);
//   main stream, beside it: pair_kernel, A -> B, the points at least 3 from
//   the edges.
// The two streams write disjoint parts of X and B and read A, X, B only where
// the other does not write, so they run concurrently; the join ends the pair.
int run_pair(lbps_lattice* lat) {
    const int a = lat->cur, b = lat->cur ^ 1;
    cudaError_t e = cudaEventRecord(lat->fork, lat->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->side, lat->fork, 0);
    if (e == cudaSuccess)
        e = lbps::with_policy(lat->p.storage, [&](auto pol) {
            using P = decltype(pol);
            const auto& g = lat->L.g;
            const auto A = lat->view<P>(a), B = lat->view<P>(b), X = lat->copy_view<P>(lat->xmem);
            // per-kernel timing: events around the two-step kernel (the passes
            // beside it are not timed, as the Newmark pass of a single step)
            cudaError_t r = prof_mark(lat);
            if (r == cudaSuccess) r = lbps::launch_pair<P>(g, lat->c, lat->kc<P>(), A, B, lat->flag(), lat->st, 32);
            if (r == cudaSuccess) r = prof_mark(lat);
            if (r == cudaSuccess && lat->prof) lat->ev_kind.push_back(0);
            auto bnd = [&](lbps::View<P> s, lbps::View<P> d, int pass) {
                return lbps::launch_boundary<P>(g, lat->c, lat->kc<P>(), s, d, lat->bn(), lat->L.nb, lat->flag(),
                                                lat->tstep(), lat->side, pass, pass + 1);
            };
            if (r == cudaSuccess) r = bnd(A, X, 1);
            if (r == cudaSuccess) r = lbps::launch_frame<P>(g, lat->c, lat->kc<P>(), A, X, lat->flag(), lat->side, 3);
            if (r == cudaSuccess) r = bnd(A, X, 2);
            if (r == cudaSuccess) r = bnd(X, B, 1);
            if (r == cudaSuccess) r = lbps::launch_frame<P>(g, lat->c, lat->kc<P>(), X, B, lat->flag(), lat->side, 2);
            if (r == cudaSuccess) r = bnd(X, B, 2);
            return r;
        });
    if (e == cudaSuccess) e = cudaEventRecord(lat->join, lat->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(lat->st, lat->join, 0);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    lat->cur = b;
    lat->steps += 2;
    return LBPS_OK;
}

// k steps: pairs in one sweep where they apply, else single steps
int run_steps(lbps_lattice* lat, int k) {
    int rc = LBPS_OK;
    for (int s = 0; s < k && rc == LBPS_OK;) {
        if (k - s >= 2 && pair_ok(lat)) {
            rc = run_pair(lat);
            s += 2;
        } else {
            rc = run_step(lat);
            s += 1;
        }
    }
    return rc;
}

void drop_graphs(lbps_lattice* lat) {
    for (int w = 0; w < 2; ++w)
        for (int q = 0; q < 2; ++q) {
            if (lat->graph[w][q]) cudaGraphExecDestroy(lat->graph[w][q]);
            lat->graph[w][q] = nullptr;
            lat->graph_gen[w][q] = -1;
        }
}

// The graph of k steps (2, or lat->graph_k) starting from the current copy:
// captured once (for the current parameters, launch shape, storage scale and
// graph_k: anything that changes them bumps lat->gen), then replayed.  The
// capture runs run_step k times on the capture stream; the host-side copy
// index and step count it advances are put back.
int step_graph(lbps_lattice* lat, int k, cudaGraphExec_t* out, int* end_cur) {
    const int q = lat->cur;
    const int w = k == 2 ? 0 : 1;
    cudaGraphExec_t& slot = lat->graph[w][q];
    if (slot && lat->graph_gen[w][q] == lat->gen) {
        *out = slot;
        *end_cur = lat->graph_cur[w][q];
        return LBPS_OK;
    }
    if (slot) cudaGraphExecDestroy(slot);
    slot = nullptr;
    if (!lat->cap && cudaStreamCreateWithFlags(&lat->cap, cudaStreamNonBlocking) != cudaSuccess) {
        lat->cap = nullptr;
        cudaGetLastError();
        return LBPS_ERR_CUDA;
    }
    cudaStream_t saved = lat->st;
    const int64_t steps = lat->steps;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(lat->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    lat->st = lat->cap;
    int rc = run_steps(lat, k);
    lat->st = saved;
    lat->graph_cur[w][q] = lat->cur;  // a pair in one sweep moves the state to the other copy once
    lat->cur = q;
    lat->steps = steps;
    e = cudaStreamEndCapture(lat->cap, &g);
    // the kernels captured from the side stream keep its priority in the graph
    if (rc == LBPS_OK && e == cudaSuccess) e = cudaGraphInstantiate(&slot, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    if (rc != LBPS_OK || e != cudaSuccess) {
        slot = nullptr;
        if (e != cudaSuccess) lat->last_cuda = (int)e;
        cudaGetLastError();
        return LBPS_ERR_CUDA;
    }
    lat->graph_gen[w][q] = lat->gen;
    *out = slot;
    *end_cur = lat->graph_cur[w][q];
    return LBPS_OK;
}

int run_sync(lbps_lattice* lat) {
    cudaError_t e = lbps::with_policy(lat->p.storage, [&](auto pol) {
        using P = decltype(pol);
        cudaError_t r = lbps::launch_sync<P>(lat->L.g, lat->c, lat->kc<P>(), lat->view<P>(lat->cur), lat->st);
        if (r == cudaSuccess)
            r = lbps::launch_mirror<P>(lat->L.g, lat->view<P>(lat->cur), lat->bn(), lat->L.nb, lat->st);
        return r;
    });
    return cuda_ok(e);
}

int run_init_kernel(lbps_lattice* lat) {
    cudaError_t e = lbps::with_policy(lat->p.storage, [&](auto pol) {
        using P = decltype(pol);
        const lbps::View<P> v = lat->view<P>(lat->cur);
        cudaError_t r = lbps::launch_init<P>(lat->L.g, lat->c, lat->kc<P>(), v, lat->st);
        if (r == cudaSuccess) r = lbps::launch_mirror<P>(lat->L.g, v, lat->bn(), lat->L.nb, lat->st);
        // the stresses of the initial u (later steps leave them with each copy)
        if (r == cudaSuccess)
            r = lbps::launch_boundary<P>(lat->L.g, lat->c, lat->kc<P>(), v, v, lat->bn(), lat->L.nb, lat->flag(),
                                         lat->tstep(), lat->st, 0, 1);
        return r;
    });
    return cuda_ok(e);
}

// 16-bit storage: the scale 2^e of the stored Nx, Ny, fixed by the
// parameters or chosen from the initial state (already in the u planes of the
// current copy) and the boundary values.
int choose_scale(lbps_lattice* lat) {
    int e = lat->p.pop_scale_exp;
    if (e == 0) {
        unsigned* word = reinterpret_cast<unsigned*>(lat->out4());
        unsigned bits = 0;
        cudaError_t ce = cudaMemsetAsync(word, 0, sizeof(unsigned), lat->st);
        if (ce == cudaSuccess)
            ce = lbps::launch_scale_probe(lat->L.g, lat->c, lat->u(lat->cur), std::sqrt(2.0 * lat->a_phi), word,
                                          lat->st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&bits, word, sizeof(bits), cudaMemcpyDeviceToHost, lat->st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(lat->st);
        if (ce != cudaSuccess) {
            lat->last_cuda = (int)ce;
            return LBPS_ERR_CUDA;
        }
        float probe;
        std::memcpy(&probe, &bits, sizeof(probe));
        double m = std::max((double)probe, lat->bc_est);
        if (m > 0.0 && std::isfinite(m)) e = 10 - (int)std::ceil(std::log2(m));
        e = std::min(100, std::max(-100, e));
    }
    lat->scale_exp = e;
    lat->kf.scale = std::ldexp(1.0f, e);
    lat->kf.inv_scale = std::ldexp(1.0f, -e);
    return LBPS_OK;
}

// Copy four [ny][nx] arrays (v may be null) into the pitched u planes of the
// copy that is not current (the current state stays intact until the input
// has been accepted).
int stage_u(lbps_lattice* lat, const double* ux0, const double* uy0, const double* vx0, const double* vy0,
            cudaMemcpyKind kind) {
    const Geo& g = lat->L.g;
    double* u = lat->u(lat->cur ^ 1);
    size_t dp = (size_t)g.px * sizeof(double), sp = (size_t)g.nx * sizeof(double);
    const double* src[4] = {ux0, uy0, vx0, vy0};
    for (int q = 0; q < 4; ++q) {
        double* dst = u + (size_t)q * g.plane;
        cudaError_t e;
        if (!src[q])
            e = cudaMemset2DAsync(dst, dp, 0, sp, g.ny, lat->st);
        else if (dp == sp)  // no row padding: one contiguous copy (a pitched one goes row by row from pageable memory)
            e = cudaMemcpyAsync(dst, src[q], sp * g.ny, kind, lat->st);
        else
            e = cudaMemcpy2DAsync(dst, dp, src[q], sp, sp, g.ny, kind, lat->st);
        if (e != cudaSuccess) return LBPS_ERR_CUDA;
    }
    return LBPS_OK;
}

// Make the staged copy current and initialise it: the initialisation kernel
// (and the 16-bit scale choice before it).
int init_staged(lbps_lattice* lat) {
    lat->cur ^= 1;
    // the non-finite flag and the step counter beside it
    if (cudaMemsetAsync(lat->flag(), 0, 16, lat->st) != cudaSuccess) return LBPS_ERR_CUDA;
    if (lat->neq16()) {
        int rc = choose_scale(lat);
        if (rc != LBPS_OK) return rc;
    }
    int rc = run_init_kernel(lat);
    if (rc != LBPS_OK) return rc;
    lat->steps = 0;
    lat->gen += 1;
    lat->initialised = true;
    return LBPS_OK;
}

size_t field_count(const lbps_lattice* lat, int32_t field) {
    size_t n = (size_t)lat->p.nx * (size_t)lat->p.ny;
    return (field == LBPS_F_PHI || field == LBPS_F_PSI) ? 5 * n : n;
}

bool valid_field(int32_t f) { return f >= LBPS_UX && f <= LBPS_STRAIN_ENERGY; }

int extract_rows(lbps_lattice* lat, int32_t field, int j0, int rows, double* dst) {
    cudaError_t e = lbps::with_policy(lat->p.storage, [&](auto pol) {
        using P = decltype(pol);
        return lbps::launch_extract_rows<P>(lat->L.g, lat->c, lat->kc<P>(), lat->view<P>(lat->cur), field, j0,
                                            rows, dst, lat->st);
    });
    return cuda_ok(e);
}

}  // namespace

extern "C" {

const char* lbps_strerror(int code) {
    switch (code) {
    case LBPS_OK: return "ok";
    case LBPS_ERR_INVALID: return "invalid argument";
    case LBPS_ERR_OOM: return "out of device memory";
    case LBPS_ERR_CUDA: return "CUDA error";
    case LBPS_ERR_NONFINITE: return "state became non-finite";
    case LBPS_ERR_TIMEOUT: return "device wait timed out";
    case LBPS_ERR_STATE: return "call out of order";
    default: return "unknown error";
    }
}

int lbps_rect_bc(int32_t nx, int32_t ny, int32_t periodic_x, int32_t periodic_y, double dh,
                 const int32_t edge_type[4], const double edge_value[8], uint8_t* node_type, double* bc_value) {
    if (nx < 3 || ny < 3 || !finite_positive(dh) || !edge_type || !edge_value || !node_type || !bc_value)
        return LBPS_ERR_INVALID;
    // edges: 0 bottom (j = 0), 1 right (i = nx-1), 2 top (j = ny-1), 3 left (i = 0)
    for (int e = 0; e < 4; ++e) {
        bool active = (e == 0 || e == 2) ? !periodic_y : !periodic_x;
        if (active && edge_type[e] != LBPS_NEUMANN && edge_type[e] != LBPS_DIRICHLET) return LBPS_ERR_INVALID;
        if (active && (!std::isfinite(edge_value[2 * e]) || !std::isfinite(edge_value[2 * e + 1])))
            return LBPS_ERR_INVALID;
    }
    for (int32_t j = 0; j < ny; ++j) {
        for (int32_t i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            bool on[4] = {!periodic_y && j == 0, !periodic_x && i == nx - 1, !periodic_y && j == ny - 1,
                          !periodic_x && i == 0};
            int n_on = 0, n_dir = 0;
            for (int e = 0; e < 4; ++e) {
                n_on += on[e];
                n_dir += on[e] && edge_type[e] == LBPS_DIRICHLET;
            }
            double vx = 0.0, vy = 0.0;
            uint8_t t = LBPS_INTERIOR;
            if (n_dir > 0) {
                // Dirichlet dominates; mean u* where two Dirichlet edges meet.
                t = LBPS_DIRICHLET;
                for (int e = 0; e < 4; ++e)
                    if (on[e] && edge_type[e] == LBPS_DIRICHLET) {
                        vx += edge_value[2 * e] / n_dir;
                        vy += edge_value[2 * e + 1] / n_dir;
                    }
            } else if (n_on > 0) {
                // Integrated traction over the external faces of the cell.
                t = LBPS_NEUMANN;
                double len = n_on == 1 ? dh : 0.5 * dh;
                for (int e = 0; e < 4; ++e)
                    if (on[e]) {
                        vx += edge_value[2 * e] * len;
                        vy += edge_value[2 * e + 1] * len;
                    }
            }
            node_type[k] = t;
            bc_value[2 * k] = vx;
            bc_value[2 * k + 1] = vy;
        }
    }
    return LBPS_OK;
}

int lbps_state_bytes(const lbps_params* params, size_t* bytes) {
    int rc = validate_params(params);
    if (rc != LBPS_OK) return rc;
    if (!bytes) return LBPS_ERR_INVALID;
    *bytes = make_layout(params).total;
    return LBPS_OK;
}

int lbps_state_bytes_cells(const lbps_params* params, const uint8_t* node_type, const double* cell, size_t* bytes) {
    int rc = validate_params(params);
    if (rc != LBPS_OK) return rc;
    if (!bytes) return LBPS_ERR_INVALID;
    if (!node_type && !cell) {  // a rectangle: the size does not depend on the node types
        *bytes = make_layout(params).total;
        return LBPS_OK;
    }
    Boundary bd;
    rc = build_boundary(params, node_type, nullptr, cell, bd);
    if (rc != LBPS_OK) return rc;
    *bytes = make_layout(params, bd.general, (int)bd.bn.size()).total;
    return LBPS_OK;
}

int lbps_create(const lbps_params* params, const uint8_t* node_type, const double* bc_value, void* device_mem,
                size_t device_bytes, lbps_lattice** out) {
    return lbps_create_cells(params, node_type, bc_value, nullptr, device_mem, device_bytes, out);
}

// Per 30-column strip of the interior kernel, the longest run of rows [a, b)
// in which none of the strip's columns holds an interior point (0, 0 if
// there is none): the rows of a hole that the interior kernel can skip.  An
// interior point's four neighbours are body points, so no interior point
// outside the run reads the populations inside it.
std::vector<int> strip_gaps(const lbps_params* p, const uint8_t* node_type) {
    const int W = lbps::kBatchStripCols;  // = the interior kernel's strip width
    const int nx = p->nx, ny = p->ny, strips = (nx + W - 1) / W;
    std::vector<int> gap(2 * (size_t)strips, 0);
    if (!node_type) return gap;
    for (int s = 0; s < strips; ++s) {
        int run = 0, best = 0, best_end = 0;
        for (int j = 0; j < ny; ++j) {
            bool any = false;
            for (int i = W * s; i < std::min(nx, W * s + W) && !any; ++i)
                any = node_type[(size_t)j * nx + i] == LBPS_INTERIOR;
            run = any ? 0 : run + 1;
            if (run > best) {
                best = run;
                best_end = j + 1;
            }
        }
        gap[2 * (size_t)s] = best_end - best;
        gap[2 * (size_t)s + 1] = best_end;
    }
    return gap;
}

int lbps_create_cells(const lbps_params* params, const uint8_t* node_type, const double* bc_value,
                      const double* cell, void* device_mem, size_t device_bytes, lbps_lattice** out) {
    if (!out) return LBPS_ERR_INVALID;
    *out = nullptr;
    int rc = validate_params(params);
    if (rc != LBPS_OK) return rc;
    Boundary bd;
    rc = build_boundary(params, node_type, bc_value, cell, bd);
    if (rc != LBPS_OK) return rc;
    Layout L = make_layout(params, bd.general, (int)bd.bn.size());
    const std::vector<BNode>& bn = bd.bn;
    lbps_lattice* lat = new (std::nothrow) lbps_lattice();
    if (!lat) return LBPS_ERR_OOM;
    lat->p = *params;
    lat->L = L;
    lat->setup_hash = setup_hash(params, bd, node_type);
    lat->st = reinterpret_cast<cudaStream_t>(params->cuda_stream);
    if (device_mem) {
        if (device_bytes < L.total || (reinterpret_cast<uintptr_t>(device_mem) % kAlign) != 0) {
            delete lat;
            return LBPS_ERR_OOM;
        }
        lat->mem = static_cast<char*>(device_mem);
        lat->owns = false;
    } else {
        if (cudaMalloc(&lat->mem, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete lat;
            return LBPS_ERR_OOM;
        }
        lat->owns = true;
    }
    // Derived constants, Eq. feq_req and Eq. conditions-parameters.
    double lam = params->lambda, mu = params->mu, rho = params->rho, dh = params->dh;
    lat->cd = std::sqrt((lam + 2.0 * mu) / rho);
    lat->cs = std::sqrt(mu / rho);
    lat->a_phi = (1.0 - params->a0_phi) / 4.0;
    lat->a_psi = (lat->cs * lat->cs) / (lat->cd * lat->cd) * lat->a_phi;
    lat->a0_psi = 1.0 - 4.0 * lat->a_psi;
    double dt = dh / lat->cd * std::sqrt(2.0 * lat->a_phi);
    Consts& c = lat->c;
    c.dt = dt;
    c.half_dt2 = 0.5 * dt * dt;
    c.lam = lam;
    c.mu = mu;
    c.rho = rho;
    c.dh = dh;
    c.inv2h = 0.5 / dh;
    c.cd2 = lat->cd * lat->cd;
    c.cs2 = lat->cs * lat->cs;
    c.a[0] = lat->a_phi;
    c.a[1] = lat->a_psi;
    c.a0[0] = params->a0_phi;
    c.a0[1] = lat->a0_psi;
    c.two_dt2 = 2.0 / (dt * dt);
    c.two_dt = 2.0 / dt;
    c.inv_rho_dh2 = 1.0 / (rho * dh * dh);
    c.bc_feq_mode = params->bc_feq_mode;
    c.bc_j_mode = params->bc_j_mode;
    // Strain scale the boundary values impose (|u*| / dh at Dirichlet points,
    // |F| / (dh mu) at Neumann points), for the 16-bit scale estimate.
    double eps = 0.0;
    for (const BNode& q : bn) {
        double m = std::max(std::fabs(q.bx), std::fabs(q.by));
        eps = std::max(eps, q.type == LBPS_DIRICHLET ? m / dh : m / (dh * mu));
    }
    lat->bc_est = std::sqrt(2.0 * lat->a_phi) * eps;
    lat->kf = make_kc<float>(lat->a_phi, lat->a_psi, c.cd2, c.cs2, dh);
    // 16-bit storage rounds its sums stochastically for slow waves (f2bits_store)
    lat->kf.sr = params->a0_phi >= kStochasticA0 ? 1u : 0u;
    lat->kd = make_kc<double>(lat->a_phi, lat->a_psi, c.cd2, c.cs2, dh);
    lat->cur = 0;
    lat->steps = 0;
    lat->initialised = false;
    // default strip height: 32 rows, or 16 / 8 where the lattice is too small
    // to give the interior kernel about 16 K warps (4-5 resident waves) at 32;
    // below about 1400^2 points a sweep of 2..16 rows (FP32, CUDA graphs) put
    // 16 rows first from about 800^2 (1024^2: 29.0 GLUPS against 25.8 at 8)
    // and 4 rows first below it (512^2: 16.4 against 15.5)
    {
        const long long strips = (params->nx + lbps::kBatchStripCols - 1) / lbps::kBatchStripCols;
        const long long points = (long long)params->nx * params->ny;
        int rows = 8;
        for (int r : {32, 16})
            if (strips * ((params->ny + r - 1) / r) >= 16384) {
                rows = r;
                break;
            }
        if (points < 640000) rows = 4;
        else if (points < 2000000) rows = 16;
        lat->tuning.rows_per_warp = rows;
        // FP64 populations need 128 registers a thread: the 6-blocks-per-SM
        // variant spills there, the 4-blocks one does not (8192^2: 12.2
        // against 9.6 GLUPS; the FP64 arithmetic bounds either)
        if (params->storage == LBPS_STORAGE_F64) lat->tuning.variant = 2;
        // BFP13's codec spills in the shape that prefetches u two rows ahead
        // at 6 blocks per SM; one row ahead fits in 80 registers
        if (params->storage == LBPS_STORAGE_BFP13) lat->tuning.variant = 4;
    }
    // the side stream of the boundary Newmark pass; if it cannot be had, the
    // pass runs on the lattice's stream (same results, no overlap).  It has
    // the greatest priority: its short dependent launches then take SM slots
    // as the interior kernel's blocks retire, instead of waiting behind all of
    // that kernel's blocks and running in its tail.
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        prio_greatest = 0;
    }
    if (cudaStreamCreateWithPriority(&lat->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&lat->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&lat->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (lat->side) cudaStreamDestroy(lat->side);
        if (lat->fork) cudaEventDestroy(lat->fork);
        if (lat->join) cudaEventDestroy(lat->join);
        lat->side = nullptr;
        lat->fork = lat->join = nullptr;
    }
    if (L.g.general) {
        lat->L.g.type = reinterpret_cast<const uint8_t*>(lat->mem + L.off_type);
        lat->L.g.gap = reinterpret_cast<const int*>(lat->mem + L.off_gap);
        lat->gap = strip_gaps(params, node_type);
    }
    cudaError_t e = cudaMemsetAsync(lat->mem, 0, L.total, lat->st);
    if (e == cudaSuccess) e = lbps::set_check_range(lat->mem, L.total, lat->st);
    if (e == cudaSuccess && L.g.general && node_type)
        e = cudaMemcpy2DAsync(lat->mem + L.off_type, (size_t)L.g.px, node_type, (size_t)L.g.nx, (size_t)L.g.nx,
                              (size_t)L.g.ny, cudaMemcpyHostToDevice, lat->st);
    if (e == cudaSuccess && L.g.general)
        e = cudaMemcpyAsync(lat->mem + L.off_gap, lat->gap.data(), lat->gap.size() * sizeof(int),
                            cudaMemcpyHostToDevice, lat->st);
    if (e == cudaSuccess && L.nb > 0)
        e = cudaMemcpyAsync(lat->mem + L.off_bn, bn.data(), bn.size() * sizeof(BNode), cudaMemcpyHostToDevice,
                            lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) {
        lbps_destroy(lat);
        return LBPS_ERR_CUDA;
    }
    *out = lat;
    return LBPS_OK;
}

int lbps_init(lbps_lattice* lat, const double* ux0, const double* uy0, const double* vx0, const double* vy0) {
    lbps::NvtxRange nvtx("lbps_init");
    if (!lat || !ux0 || !uy0 || (!vx0) != (!vy0)) return LBPS_ERR_INVALID;
    int rc = stage_u(lat, ux0, uy0, vx0, vy0, cudaMemcpyHostToDevice);
    if (rc != LBPS_OK) return rc;
    // finiteness of the input, checked on the device over the staged planes
    unsigned* bad = reinterpret_cast<unsigned*>(lat->out4());
    unsigned h_bad = 0;
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), lat->st);
    if (e == cudaSuccess) e = lbps::launch_finite_check(lat->L.g, lat->u(lat->cur ^ 1), vx0 ? 4 : 2, bad, lat->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    if (h_bad) {
        // rejected: the current state is untouched; clear the staging planes
        // (points a step never writes, such as void points, must stay zero)
        e = cudaMemsetAsync(lat->u(lat->cur ^ 1), 0, lat->L.u_bytes, lat->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
        if (e != cudaSuccess) {
            lat->last_cuda = (int)e;
            return LBPS_ERR_CUDA;
        }
        return LBPS_ERR_INVALID;
    }
    rc = init_staged(lat);
    if (rc != LBPS_OK) return rc;
    e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) lat->last_cuda = (int)e;
    return cuda_ok(e);
}

int lbps_init_device(lbps_lattice* lat, const double* d_ux0, const double* d_uy0, const double* d_vx0,
                     const double* d_vy0) {
    lbps::NvtxRange nvtx("lbps_init_device");
    if (!lat || !d_ux0 || !d_uy0 || (!d_vx0) != (!d_vy0)) return LBPS_ERR_INVALID;
    int rc = stage_u(lat, d_ux0, d_uy0, d_vx0, d_vy0, cudaMemcpyDeviceToDevice);
    if (rc != LBPS_OK) return rc;
    return init_staged(lat);
}

int lbps_step_async(lbps_lattice* lat, int64_t n) {
    lbps::NvtxRange nvtx("lbps_step_async");
    if (!lat || n < 0) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    if (n >= 2 && solo_pairs(lat)) {
        if (!lat->solo) {
            lbps_lattice* one = lat;
            int rc = lbps_batch_create(&one, 1, lat->st, &lat->solo);
            if (rc == LBPS_OK) rc = lbps_batch_set_step_pairs(lat->solo, 1);
            if (rc != LBPS_OK) {
                drop_solo(lat);
                return rc;
            }
        }
        return lbps_batch_step(lat->solo, n);
    }
    const int l = lat->p.sync_every;
    for (int64_t s = 0; s < n;) {
        // graph_k steps at once from a graph, else 2, unless per-kernel timing
        // is on or a synchronisation falls after one of the first k - 1 of them
        int k = 0;
        for (int c : {lat->graph_k, 2})
            if (k == 0 && n - s >= c && !lat->prof && !(l > 0 && l - lat->steps % l < c)) k = c;
        if (k > 0) {
            cudaGraphExec_t g = nullptr;
            int end_cur = lat->cur;
            int rc = step_graph(lat, k, &g, &end_cur);
            if (rc != LBPS_OK) return rc;
            cudaError_t e = cudaGraphLaunch(g, lat->st);
            if (e != cudaSuccess) {
                lat->last_cuda = (int)e;
                return LBPS_ERR_CUDA;
            }
            lat->steps += k;
            lat->cur = end_cur;
            s += k;
        } else if (n - s >= 2 && pair_ok(lat) && !(l > 0 && (lat->steps + 1) % l == 0)) {
            int rc = run_pair(lat);
            if (rc != LBPS_OK) return rc;
            s += 2;
        } else {
            int rc = run_step(lat);
            if (rc != LBPS_OK) return rc;
            s += 1;
        }
        if (l > 0 && lat->steps % l == 0) {
            int rc = run_sync(lat);
            if (rc != LBPS_OK) return rc;
        }
    }
    return LBPS_OK;
}

int lbps_check(lbps_lattice* lat) {
    if (!lat) return LBPS_ERR_INVALID;
    unsigned flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, lat->flag(), sizeof(unsigned), cudaMemcpyDeviceToHost, lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    return flag ? LBPS_ERR_NONFINITE : LBPS_OK;
}

int lbps_step(lbps_lattice* lat, int64_t n) {
    int rc = lbps_step_async(lat, n);
    if (rc != LBPS_OK) return rc;
    return lbps_check(lat);
}

int lbps_sync(lbps_lattice* lat) {
    lbps::NvtxRange nvtx("lbps_sync");
    if (!lat) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    return run_sync(lat);
}

int lbps_read_device(lbps_lattice* lat, int32_t field, double* d_dst, size_t count) {
    lbps::NvtxRange nvtx("lbps_read_device");
    if (!lat || !d_dst || !valid_field(field)) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    if (count < field_count(lat, field)) return LBPS_ERR_INVALID;
    return extract_rows(lat, field, 0, lat->p.ny, d_dst);
}

int lbps_read(lbps_lattice* lat, int32_t field, double* dst, size_t count) {
    lbps::NvtxRange nvtx("lbps_read");
    if (!lat || !dst || !valid_field(field)) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    if (count < field_count(lat, field)) return LBPS_ERR_INVALID;
    const Geo& g = lat->L.g;
    size_t nx = (size_t)g.nx, n = nx * (size_t)g.ny;
    if (field >= LBPS_UX && field <= LBPS_VY && (size_t)g.px == nx) {
        // a stored plane without row padding: one contiguous copy
        cudaError_t e = cudaMemcpyAsync(dst, lat->u(lat->cur) + (size_t)field * g.plane, n * sizeof(double),
                                        cudaMemcpyDeviceToHost, lat->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
        if (e != cudaSuccess) {
            lat->last_cuda = (int)e;
            return LBPS_ERR_CUDA;
        }
        return LBPS_OK;
    }
    int planes = (field == LBPS_F_PHI || field == LBPS_F_PSI) ? 5 : 1;
    size_t row_bytes = (size_t)planes * nx * sizeof(double);
    int chunk = (int)(lat->L.staging_bytes / row_bytes);
    if (chunk < 1) return LBPS_ERR_INVALID;
    double* stg = lat->staging();
    for (int j0 = 0; j0 < g.ny; j0 += chunk) {
        int rows = g.ny - j0 < chunk ? g.ny - j0 : chunk;
        int rc = extract_rows(lat, field, j0, rows, stg);
        if (rc != LBPS_OK) return rc;
        for (int q = 0; q < planes; ++q) {
            cudaError_t e = cudaMemcpyAsync(dst + (size_t)q * n + (size_t)j0 * nx, stg + (size_t)q * rows * nx,
                                            (size_t)rows * nx * sizeof(double), cudaMemcpyDeviceToHost, lat->st);
            if (e != cudaSuccess) return LBPS_ERR_CUDA;
        }
        // no wait here: the next chunk's kernel runs after this copy on the stream
    }
    if (cudaStreamSynchronize(lat->st) != cudaSuccess) return LBPS_ERR_CUDA;
    return LBPS_OK;
}

int lbps_norms(lbps_lattice* lat, int32_t field, const double* d_ref, double out[4]) {
    lbps::NvtxRange nvtx("lbps_norms");
    if (!lat || !out) return LBPS_ERR_INVALID;
    if (!(field >= LBPS_UX && field <= LBPS_PSI) && !(field >= LBPS_CONSISTENCY && field <= LBPS_STRAIN_ENERGY))
        return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    cudaError_t e = lbps::with_policy(lat->p.storage, [&](auto pol) {
        using P = decltype(pol);
        return lbps::launch_norms<P>(lat->L.g, lat->c, lat->kc<P>(), lat->view<P>(lat->cur), field, d_ref,
                                     lat->partials(), lat->out4(), lat->st);
    });
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, lat->out4(), 4 * sizeof(double), cudaMemcpyDeviceToHost, lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    return cuda_ok(e);
}

int lbps_energy(lbps_lattice* lat, double out[3]) {
    lbps::NvtxRange nvtx("lbps_energy");
    if (!lat || !out) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    double n[2][4];
    for (int q = 0; q < 2; ++q) {
        int rc = lbps_norms(lat, q == 0 ? LBPS_KINETIC_ENERGY : LBPS_STRAIN_ENERGY, nullptr, n[q]);
        if (rc != LBPS_OK) return rc;
    }
    const double area = lat->p.dh * lat->p.dh;
    out[0] = n[0][2] * area;
    out[1] = n[1][2] * area;
    out[2] = out[0] + out[1];
    return LBPS_OK;
}

int lbps_info(const lbps_lattice* lat, double out[6], int64_t* steps_done) {
    if (!lat) return LBPS_ERR_INVALID;
    if (out) {
        out[0] = lat->cd;
        out[1] = lat->cs;
        out[2] = lat->a_phi;
        out[3] = lat->a_psi;
        out[4] = lat->a0_psi;
        out[5] = lat->c.dt;
    }
    if (steps_done) *steps_done = lat->steps;
    return LBPS_OK;
}

namespace {

// Header of a saved state; the raw current state copy follows it.
struct SavedState {
    char magic[8];          // "LBPSSTA2"
    int32_t nx, ny, px, storage;
    int32_t scale_exp, pad;
    int64_t steps;
    uint64_t copy_bytes;
    uint64_t setup_hash;    // parameters and boundary description of the saving lattice
};

constexpr char kMagic[8] = {'L', 'B', 'P', 'S', 'S', 'T', 'A', '2'};

}  // namespace

int lbps_state_size(const lbps_lattice* lat, size_t* bytes) {
    if (!lat || !bytes) return LBPS_ERR_INVALID;
    *bytes = sizeof(SavedState) + lat->L.copy_bytes;
    return LBPS_OK;
}

int lbps_state_save(lbps_lattice* lat, void* dst, size_t bytes) {
    lbps::NvtxRange nvtx("lbps_state_save");
    if (!lat || !dst || bytes < sizeof(SavedState) + lat->L.copy_bytes) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    SavedState h{};
    std::memcpy(h.magic, kMagic, sizeof(kMagic));
    h.nx = lat->L.g.nx;
    h.ny = lat->L.g.ny;
    h.px = lat->L.g.px;
    h.storage = lat->p.storage;
    h.scale_exp = lat->scale_exp;
    h.steps = lat->steps;
    h.copy_bytes = lat->L.copy_bytes;
    h.setup_hash = lat->setup_hash;
    // dst may be host or device memory: both copies go through the runtime
    cudaError_t e = cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyDefault, lat->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(static_cast<char*>(dst) + sizeof(h), lat->mem + lat->L.off_copy[lat->cur],
                            lat->L.copy_bytes, cudaMemcpyDefault, lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    return LBPS_OK;
}

int lbps_state_load(lbps_lattice* lat, const void* src, size_t bytes) {
    lbps::NvtxRange nvtx("lbps_state_load");
    if (!lat || !src || bytes < sizeof(SavedState)) return LBPS_ERR_INVALID;
    SavedState h;
    // src may be host or device memory
    cudaError_t he = cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, lat->st);
    if (he == cudaSuccess) he = cudaStreamSynchronize(lat->st);
    if (he != cudaSuccess) {
        lat->last_cuda = (int)he;
        return LBPS_ERR_CUDA;
    }
    if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0 || h.nx != lat->L.g.nx || h.ny != lat->L.g.ny ||
        h.px != lat->L.g.px || h.storage != lat->p.storage || h.copy_bytes != lat->L.copy_bytes ||
        bytes < sizeof(SavedState) + lat->L.copy_bytes || h.steps < 0 || h.scale_exp < -100 || h.scale_exp > 100 ||
        h.setup_hash != lat->setup_hash)
        return LBPS_ERR_INVALID;
    lat->cur = 0;
    cudaError_t e = cudaMemcpyAsync(lat->mem + lat->L.off_copy[0], static_cast<const char*>(src) + sizeof(h),
                                    lat->L.copy_bytes, cudaMemcpyDefault, lat->st);
    unsigned long long n = (unsigned long long)h.steps;
    // the non-finite flag cleared, the device step counter set
    if (e == cudaSuccess) e = cudaMemsetAsync(lat->flag(), 0, sizeof(unsigned), lat->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lat->tstep(), &n, sizeof(n), cudaMemcpyHostToDevice, lat->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->st);
    if (e != cudaSuccess) {
        lat->last_cuda = (int)e;
        return LBPS_ERR_CUDA;
    }
    lat->steps = h.steps;
    lat->scale_exp = h.scale_exp;
    lat->kf.scale = std::ldexp(1.0f, h.scale_exp);
    lat->kf.inv_scale = std::ldexp(1.0f, -h.scale_exp);
    lat->initialised = true;
    lat->gen += 1;  // batches holding this lattice re-read its descriptor
    return LBPS_OK;
}

int lbps_set_load(lbps_lattice* lat, int32_t kind, double t_ramp, double t_hold) {
    if (!lat || (kind != LBPS_NEUMANN && kind != LBPS_DIRICHLET)) return LBPS_ERR_INVALID;
    if (!(t_ramp >= 0.0) || !std::isfinite(t_ramp) || !(t_hold > 0.0)) return LBPS_ERR_INVALID;
    const int q = kind == LBPS_NEUMANN ? 0 : 1;
    lat->c.load_rate[q] = t_ramp > 0.0 ? 1.0 / t_ramp : 0.0;
    lat->c.load_hold[q] = t_hold;
    lat->gen += 1;  // batches holding this lattice re-read its descriptor
    return LBPS_OK;
}

int lbps_scale_exp(const lbps_lattice* lat, int32_t* exp) {
    if (!lat || !exp) return LBPS_ERR_INVALID;
    *exp = lat->neq16() ? lat->scale_exp : 0;
    return LBPS_OK;
}

int lbps_last_cuda_error(const lbps_lattice* lat) { return lat ? lat->last_cuda : 0; }

int lbps_check_report(uint64_t out[2]) {
    if (!out) return LBPS_ERR_INVALID;
    unsigned long long r[2] = {0, 0};
    int rc = lbps::check_report(r);
    out[0] = r[0];
    out[1] = r[1];
    return rc < 0 ? LBPS_ERR_CUDA : rc;
}

int lbps_set_tuning(lbps_lattice* lat, int32_t variant, int32_t rows_per_warp) {
    if (!lat || variant < 0 || variant >= lbps::kTuningVariants || rows_per_warp < 1 || rows_per_warp > 4096)
        return LBPS_ERR_INVALID;
    lat->tuning.variant = variant;
    lat->tuning.rows_per_warp = rows_per_warp;
    lat->gen += 1;  // captured step graphs use the old launch shape
    return LBPS_OK;
}

int lbps_set_step_pairs(lbps_lattice* lat, int32_t on) {
    if (!lat || on < 0 || on > 1) return LBPS_ERR_INVALID;
    if ((on != 0) == (lat->xmem != nullptr)) return LBPS_OK;
    if (cudaStreamSynchronize(lat->st) != cudaSuccess) return LBPS_ERR_CUDA;
    drop_solo(lat);
    if (on) {
        void* x = nullptr;
        if (cudaMalloc(&x, lat->L.copy_bytes) != cudaSuccess) {
            cudaGetLastError();
            return LBPS_ERR_OOM;
        }
        // zeroed once: parts of it the frame passes read but do not use then hold finite values
        if (cudaMemset(x, 0, lat->L.copy_bytes) != cudaSuccess ||
            lbps::set_check_range(x, lat->L.copy_bytes, lat->st) != cudaSuccess) {
            cudaFree(x);
            cudaGetLastError();
            return LBPS_ERR_CUDA;
        }
        lat->xmem = static_cast<char*>(x);
    } else {
        lbps::set_check_range(lat->xmem, 0, lat->st);
        cudaFree(lat->xmem);
        lat->xmem = nullptr;
    }
    lat->gen += 1;  // captured step graphs hold the other kind of step
    return LBPS_OK;
}

int lbps_step_pairs(const lbps_lattice* lat) {
    if (!lat) return LBPS_ERR_INVALID;
    return pair_ok(lat) ? 1 : 0;
}

int lbps_set_graph_steps(lbps_lattice* lat, int32_t k) {
    if (!lat || k < 2 || k > 64 || (k & 1)) return LBPS_ERR_INVALID;
    lat->graph_k = k;
    lat->gen += 1;  // captured step graphs hold the old number of steps
    return LBPS_OK;
}

int lbps_profile(lbps_lattice* lat, int32_t enable) {
    if (!lat) return LBPS_ERR_INVALID;
    lat->prof = enable != 0;
    return LBPS_OK;
}

int lbps_profile_read(lbps_lattice* lat, double out[4]) {
    if (!lat || !out) return LBPS_ERR_INVALID;
    if (cudaStreamSynchronize(lat->st) != cudaSuccess) return LBPS_ERR_CUDA;
    for (int q = 0; q < 4; ++q) out[q] = 0.0;
    for (size_t r = 0; r < lat->ev_kind.size(); ++r) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, lat->ev_pool[2 * r], lat->ev_pool[2 * r + 1]) != cudaSuccess)
            return LBPS_ERR_CUDA;
        int k = lat->ev_kind[r];
        out[2 * k] += ms;
        out[2 * k + 1] += 1.0;
    }
    lat->ev_kind.clear();
    lat->ev_used = 0;
    return LBPS_OK;
}

// ---- rows of the state for a domain decomposition

namespace {

// The copy of rows [row0, row0 + rows) of every plane of the current state
// (populations in the storage layout, then u_x, u_y, v_x, v_y) to or from
// buf, plane after plane, each rows x px elements (row padding included).
int halo_segments(lbps_lattice* lat, int32_t row0, int32_t rows, char* buf, bool pack, lbps::CopySegs& s) {
    const Layout& L = lat->L;
    const size_t px = (size_t)L.g.px;
    const size_t base = lbps::with_policy(lat->p.storage, [](auto pol) { return sizeof(typename decltype(pol)::Base); });
    const int planes = lbps::with_policy(lat->p.storage, [](auto pol) { return decltype(pol)::kBytesPerPoint; }) /
                       (int)base;
    if (planes + 4 > lbps::kMaxCopySegs) return LBPS_ERR_INVALID;
    char* copy = lat->mem + L.off_copy[lat->cur];
    char* u = reinterpret_cast<char*>(lat->u(lat->cur));
    size_t off = 0;
    s.n = 0;
    s.pack = pack ? 1 : 0;
    auto add = [&](char* lattice_side, size_t bytes) {
        s.src[s.n] = pack ? lattice_side : buf + off;
        s.dst[s.n] = pack ? buf + off : lattice_side;
        s.bytes[s.n] = bytes;
        ++s.n;
        off += bytes;
    };
    for (int q = 0; q < planes; ++q) add(copy + ((size_t)q * L.g.plane + (size_t)row0 * px) * base, (size_t)rows * px * base);
    for (int q = 0; q < 4; ++q) add(u + ((size_t)q * L.g.plane + (size_t)row0 * px) * sizeof(double), (size_t)rows * px * 8);
    return LBPS_OK;
}

size_t halo_bytes_of(const lbps_lattice* lat, int32_t rows) {
    const size_t per = lbps::with_policy(lat->p.storage, [](auto pol) { return (size_t)decltype(pol)::kBytesPerPoint; });
    return (size_t)rows * (size_t)lat->L.g.px * (per + 32);
}

int halo_check(const lbps_lattice* lat, int32_t row0, int32_t rows, const void* buf, size_t bytes) {
    if (!lat || !buf || rows < 1 || row0 < 0 || row0 + rows > lat->L.g.ny) return LBPS_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(buf) % 16 != 0 || bytes < halo_bytes_of(lat, rows)) return LBPS_ERR_INVALID;
    if (!lat->initialised) return LBPS_ERR_STATE;
    return LBPS_OK;
}

}  // namespace

int lbps_halo_bytes(const lbps_lattice* lat, int32_t rows, size_t* bytes) {
    if (!lat || !bytes || rows < 1 || rows > lat->L.g.ny) return LBPS_ERR_INVALID;
    *bytes = halo_bytes_of(lat, rows);
    return LBPS_OK;
}

int lbps_halo_pack(lbps_lattice* lat, int32_t row0, int32_t rows, void* d_buf, size_t bytes) {
    lbps::NvtxRange nvtx("lbps_halo_pack");
    int rc = halo_check(lat, row0, rows, d_buf, bytes);
    if (rc != LBPS_OK) return rc;
    lbps::CopySegs s;
    rc = halo_segments(lat, row0, rows, static_cast<char*>(d_buf), true, s);
    if (rc != LBPS_OK) return rc;
    cudaError_t e = lbps::launch_copy_segments(s, lat->st);
    if (e != cudaSuccess) lat->last_cuda = (int)e;
    return cuda_ok(e);
}

int lbps_halo_unpack(lbps_lattice* lat, int32_t row0, int32_t rows, const void* d_buf, size_t bytes) {
    lbps::NvtxRange nvtx("lbps_halo_unpack");
    int rc = halo_check(lat, row0, rows, d_buf, bytes);
    if (rc != LBPS_OK) return rc;
    lbps::CopySegs s;
    rc = halo_segments(lat, row0, rows, const_cast<char*>(static_cast<const char*>(d_buf)), false, s);
    if (rc != LBPS_OK) return rc;
    cudaError_t e = lbps::launch_copy_segments(s, lat->st);
    // the copy's derived boundary data: stresses of its u and the boundary mirror
    if (e == cudaSuccess)
        e = lbps::with_policy(lat->p.storage, [&](auto pol) {
            using P = decltype(pol);
            const lbps::View<P> v = lat->view<P>(lat->cur);
            cudaError_t r = lbps::launch_mirror<P>(lat->L.g, v, lat->bn(), lat->L.nb, lat->st);
            if (r == cudaSuccess)
                r = lbps::launch_boundary<P>(lat->L.g, lat->c, lat->kc<P>(), v, v, lat->bn(), lat->L.nb, lat->flag(),
                                             lat->tstep(), lat->st, 0, 1);
            return r;
        });
    if (e != cudaSuccess) lat->last_cuda = (int)e;
    return cuda_ok(e);
}

int lbps_set_origin(lbps_lattice* lat, int64_t row0) {
    if (!lat) return LBPS_ERR_INVALID;
    lat->kf.key4 = (unsigned)((uint64_t)row0 * (uint64_t)lat->L.g.px * 4u);
    lat->gen += 1;  // batches holding this lattice re-read its descriptor
    return LBPS_OK;
}

int lbps_set_stream(lbps_lattice* lat, void* cuda_stream) {
    if (!lat) return LBPS_ERR_INVALID;
    lat->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    lat->p.cuda_stream = cuda_stream;
    return LBPS_OK;
}

void lbps_destroy(lbps_lattice* lat) {
    if (!lat) return;
    drop_solo(lat);
    drop_graphs(lat);
    if (lat->cap) cudaStreamDestroy(lat->cap);
    if (lat->side) {
        cudaStreamSynchronize(lat->side);
        cudaStreamDestroy(lat->side);
    }
    if (lat->fork) cudaEventDestroy(lat->fork);
    if (lat->join) cudaEventDestroy(lat->join);
    if (lat->mem) lbps::set_check_range(lat->mem, 0, lat->st);  // checked builds: the block is no longer live
    if (lat->xmem) {
        lbps::set_check_range(lat->xmem, 0, lat->st);
        cudaStreamSynchronize(lat->st);
        cudaFree(lat->xmem);
    }
    if (lat->owns && lat->mem) {
        cudaStreamSynchronize(lat->st);
        cudaFree(lat->mem);
    }
    for (cudaEvent_t e : lat->ev_pool) cudaEventDestroy(e);
    delete lat;
}

}  // extern "C"
