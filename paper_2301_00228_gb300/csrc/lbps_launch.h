// Host-side launchers of the LBM kernels (defined in lbps_kernels.cu).
#pragma once

#include "lbps_device.cuh"

namespace lbps {

template <typename T>
cudaError_t launch_init(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, const double* ux0,
                        const double* uy0, const double* vx0, const double* vy0, cudaStream_t st);

// One time step A (time t) -> B (time t + dt) on one stream: boundary passes
// 0-1 (stress, Newmark), launch_bulk, boundary pass 2 (reset).  sig: scratch
// of 2 * nb * 3 doubles (stresses of the boundary cells).
template <typename T>
cudaError_t launch_boundary(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B,
                            const BNode* bn, int nb, double* sig, unsigned* flag, cudaStream_t st, int pass_lo,
                            int pass_hi);
// Launch shape of the bulk kernel: variant selects the register budget (0: 6
// blocks of 128 threads per SM, 1: 5, 2: 4, 3: 8), rows_per_warp the height of
// the strip each warp marches over.  Results do not depend on either.
struct Tuning {
    int variant = 0;
    int rows_per_warp = 32;
};
constexpr int kTuningVariants = 4;
template <typename T>
cudaError_t launch_bulk(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, View<T> B, unsigned* flag,
                        cudaStream_t st, const Tuning& tu);

template <typename T>
cudaError_t launch_sync(const Geo& g, const Consts& c, const KC<T>& k, View<T> A, cudaStream_t st);

// Dense FP64 copy of one field (ids of lbps.h).
template <typename T>
cudaError_t launch_extract(const Geo& g, const Consts& c, View<T> A, int field, double* dst, cudaStream_t st);

// Rows [j0, j0 + rows) only, into a dense [rows][nx] (x5 for populations) buffer.
template <typename T>
cudaError_t launch_extract_rows(const Geo& g, const Consts& c, View<T> A, int field, int j0, int rows,
                                double* dst, cudaStream_t st);

// FP64 reductions of one scalar field against an optional reference;
// partials: scratch of at least kNormBlocks * 4 doubles.
constexpr int kNormBlocks = 1024;
template <typename T>
cudaError_t launch_norms(const Geo& g, const Consts& c, View<T> A, int field, const double* ref,
                         double* partials, double* out4, cudaStream_t st);

// ---- batches: many lattices advanced by one launch of each kernel per step

// Everything the kernels need about one lattice of a batch.  v[cur] holds the
// state at the start of a batch step pair; a step with parity p reads
// v[cur ^ p] and writes v[cur ^ p ^ 1].
template <typename T>
struct DomDesc {
    Geo g;
    Consts c;
    KC<T> k;
    View<T> v[2];
    const BNode* bn;
    double* sig;
    unsigned* flag;
    int nb;
    int cur;
};

struct BulkTask {  // one warp: output columns [xs, xs + 30) of rows [j0, j1) of lattice dom
    int dom, xs, j0, j1;
};

struct BndTask {   // one thread: boundary point b of lattice dom
    int dom, b;
};

constexpr int kBatchStripCols = 30;  // output columns per warp task

template <typename T>
cudaError_t launch_boundary_batch(const DomDesc<T>* dd, const BndTask* tasks, int ntasks, int parity, int pass_lo,
                                  int pass_hi, cudaStream_t st);
template <typename T>
cudaError_t launch_bulk_batch(const DomDesc<T>* dd, const BulkTask* tasks, int ntasks, int parity, int variant,
                              cudaStream_t st);

// Checked builds (LBPS_CHECKED): the device block every kernel access must
// stay inside, and the first violation seen (source line, address); both are
// no-ops returning 0 in normal builds.
cudaError_t set_check_range(const void* base, size_t bytes, cudaStream_t st);
int check_report(unsigned long long out[2]);

}  // namespace lbps
