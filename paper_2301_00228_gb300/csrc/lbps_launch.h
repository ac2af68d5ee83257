// Host-side launchers of the LBM kernels (defined in lbps_kernels.cu).
#pragma once

#include "lbps_device.cuh"

namespace lbps {

template <typename P>
using KCof = KC<typename P::V>;

// The storage policies the library is built for (lbps_device.cuh), by
// LBPS_STORAGE_* code.
using PolF32 = PopDirect<float>;
using PolF64 = PopDirect<double>;
using PolBF16 = PopNeq16<__nv_bfloat16>;
using PolF16 = PopNeq16<__half>;
using PolBfp13 = PopBfp13;

// *bad |= 1 if one of the first `planes` u planes holds a non-finite value at
// a lattice point (zero *bad first).
cudaError_t launch_finite_check(const Geo& g, const double* u, int planes, unsigned* bad, cudaStream_t st);

// Largest per-point estimate of |J| (scale_probe_kernel): FP32 bits
// of a non-negative value, atomically maxed into *out (zero it first).
cudaError_t launch_scale_probe(const Geo& g, const Consts& c, const double* u, double sq, unsigned* out,
                               cudaStream_t st);

template <typename P>
cudaError_t launch_init(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, cudaStream_t st);
// Refreshes A's boundary mirror from the lattice (after launch_init and
// launch_sync, which write boundary populations in place).
template <typename P>
cudaError_t launch_mirror(const Geo& g, View<P> A, const BNode* bn, int nb, cudaStream_t st);

// One time step A (time t) -> B (time t + dt) on one stream: boundary pass 1
// (Newmark, from A's stresses), launch_bulk, boundary pass 2 (reset, which
// also writes B's stresses).  Pass 0 computes A's stresses from A's u, for
// a copy whose u was set otherwise (initialisation).  tstep: the lattice's
// step counter, read by pass 1 and advanced by pass 2.
template <typename P>
cudaError_t launch_boundary(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B,
                            const BNode* bn, int nb, unsigned* flag, unsigned long long* tstep,
                            cudaStream_t st, int pass_lo, int pass_hi);
// Launch shape of the bulk kernel: variant selects the register budget (0: 6
// blocks of 128 threads per SM, 1: 5, 2: 4, 3: 8) with u, du/dt prefetched two
// rows ahead like the populations; variants 4..7 the same budgets with u,
// du/dt one row ahead (fewer registers, less memory in flight).
// rows_per_warp is the height of the strip each warp marches over.  Results
// do not depend on either.
struct Tuning {
    int variant = 0;
    int rows_per_warp = 32;
};
constexpr int kTuningVariants = 8;
template <typename P>
cudaError_t launch_bulk(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                        cudaStream_t st, const Tuning& tu);
// Two steps per sweep of a rectangle without periodic axes (min side >= 16):
// launch_pair writes step n + 2 of the points at least 3 from every edge
// (copy A holds step n); launch_frame runs the interior kernel on the points
// 1 .. fw from the edges only (four bands).
template <typename P>
cudaError_t launch_pair(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                        cudaStream_t st, int rows);
template <typename P>
cudaError_t launch_frame(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, View<P> B, unsigned* flag,
                         cudaStream_t st, int fw);

template <typename P>
cudaError_t launch_sync(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, cudaStream_t st);

// Rows [j0, j0 + rows) of one field (ids of lbps.h) into a dense FP64
// [rows][nx] (x5 for populations) buffer.
template <typename P>
cudaError_t launch_extract_rows(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, int field, int j0,
                                int rows, double* dst, cudaStream_t st);

// FP64 reductions of one scalar field against an optional reference;
// partials: scratch of at least kNormBlocks * 4 doubles.
constexpr int kNormBlocks = 1024;
template <typename P>
cudaError_t launch_norms(const Geo& g, const Consts& c, const KCof<P>& k, View<P> A, int field, const double* ref,
                         double* partials, double* out4, cudaStream_t st);

// ---- batches: many lattices advanced by one launch of each kernel per step

// Everything the kernels need about one lattice of a batch.  v[cur] holds the
// state at the start of a batch step pair; a step with parity p reads
// v[cur ^ p] and writes v[cur ^ p ^ 1].
template <typename P>
struct DomDesc {
    Geo g;
    Consts c;
    KCof<P> k;
    View<P> v[2];
    View<P> x;  // scratch state copy of two steps per sweep (unset without)
    const BNode* bn;
    unsigned* flag;
    unsigned long long* tstep;  // step counter (time of the boundary data)
    int nb;
    int cur;
};

struct BulkTask {  // one warp: output columns [xs, xs + 30) of rows [j0, j1) of lattice dom;
    int dom, xs, j0, j1;  // j0 < 0: the Newmark pass of boundary tasks [xs, xs + j1), j1 <= 32
};

struct BndTask {   // one thread: boundary point b of lattice dom
    int dom, b;
};

// One warp's task of the two-steps-per-sweep batch kernel: kind kPairStrip,
// output columns [xs, xs + 28) of rows [j0, j1) of lattice dom advanced two
// steps; kFrameStrip, the interior kernel on strip xs, rows [j0, j1), writing
// only inside the window [x0, x1) x [y0, y1); kNewmarkTask, the Newmark pass
// of boundary tasks [xs, xs + j1).
constexpr int kPairStrip = 0;
constexpr int kFrameStrip = 1;
constexpr int kNewmarkTask = 2;
struct PairTask {
    int dom, kind, xs, j0, j1;
    int x0, x1, y0, y1;
};

constexpr int kBatchStripCols = 30;  // output columns per warp task

// stage 0: copy v[a] -> v[a ^ 1] (a = cur ^ parity); with two steps per
// sweep, stage 1: v[a] -> x and stage 2: x -> v[a ^ 1].
template <typename P>
cudaError_t launch_boundary_batch(const DomDesc<P>* dd, const BndTask* tasks, int ntasks, int parity, int pass_lo,
                                  int pass_hi, cudaStream_t st, int stage = 0);
// One stage of a pair of steps of every lattice (two steps per sweep): a
// persistent grid whose warps take PairTasks through the counter *next
// (zeroed by the caller).  Stage 1: two-step strips v[a] -> v[a ^ 1], frame
// strips and Newmark tasks v[a] -> x; stage 2: frame strips and Newmark tasks
// x -> v[a ^ 1].
template <typename P>
cudaError_t launch_pair_batch(const DomDesc<P>* dd, const PairTask* tasks, int ntasks, const BndTask* btasks,
                              int parity, int stage, unsigned* next, cudaStream_t st);
// Interior of every lattice and the Newmark pass of their boundary points: a
// persistent grid whose warps take tasks (strips, or 32 boundary points of
// btasks) through the counter *next (device memory; the launcher zeroes it on
// the stream).
template <typename P>
cudaError_t launch_bulk_batch(const DomDesc<P>* dd, const BulkTask* tasks, int ntasks, const BndTask* btasks,
                              int parity, int variant, unsigned* next, cudaStream_t st);

// Rows of a state copy to or from a caller buffer (domain decomposition):
// up to kMaxCopySegs contiguous byte ranges, each a multiple of 16 bytes and
// 16-byte aligned at both ends.  pack: lattice -> buffer; otherwise buffer ->
// lattice.
constexpr int kMaxCopySegs = 16;
struct CopySegs {
    const char* src[kMaxCopySegs];
    char* dst[kMaxCopySegs];
    size_t bytes[kMaxCopySegs];
    int n;
    int pack;
};
cudaError_t launch_copy_segments(const CopySegs& s, cudaStream_t st);

// Checked builds (LBPS_CHECKED): set_check_range adds a live lattice block
// that kernel accesses may touch (bytes = 0 removes the block starting at
// base); check_report returns the first violation since the library was
// loaded (source line, address).  Both are no-ops returning 0 in normal
// builds.
cudaError_t set_check_range(const void* base, size_t bytes, cudaStream_t st);
int check_report(unsigned long long out[2]);

}  // namespace lbps
