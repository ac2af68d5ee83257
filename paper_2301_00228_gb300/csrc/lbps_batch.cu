// Batches of lattices (lbps_batch_* in include/lbps.h): every lattice of a
// batch advances by two launches per time step, the persistent kernel (the
// interior strips and the boundary Newmark pass of every lattice, from one
// device-side work list) and the boundary reset; blocks of k steps (k even,
// tuned) are captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lbps.h"
#include "lbps_launch.h"
#include "lbps_state.h"

using lbps::BndTask;
using lbps::BulkTask;
using lbps::DomDesc;
using lbps::PairTask;

struct lbps_batch {
    std::vector<lbps_lattice*> lats;
    int32_t storage = LBPS_STORAGE_F32;
    cudaStream_t st = nullptr;    // stream the graph runs on
    bool own_stream = false;
    char* mem = nullptr;          // descriptors | boundary tasks | bulk tasks
    size_t mem_bytes = 0;
    size_t off_bnd = 0, off_bulk = 0, off_next = 0;
    int nbnd = 0, nbulk = 0;
    size_t max_bulk = 0;  // capacity of the device work list (tasks)
    // default launch shape: 5 blocks per SM (no spills in the batched
    // kernel), u one row ahead, 16-row chunks; the fastest or within 3 % of
    // it on mixed batches of 64-2048-point sides (lbps_batch_tune refines it)
    int variant = 5, rows = 16;
    int graph_k = 2;              // steps per replayed graph (even)
    std::vector<int> uploaded_cur;
    std::vector<int64_t> uploaded_gen;
    cudaGraphExec_t graph = nullptr;    // graph_k steps
    cudaGraphExec_t pair = nullptr;     // 2 steps (what is left of n after the k-step blocks)
    cudaEvent_t order = nullptr;  // orders the batch stream with the lattices' streams
    int last_cuda = 0;
    // two steps per sweep (lbps_batch_set_step_pairs): the task lists of the
    // two stages of a pair, stage 1 then stage 2, in their own device block
    bool pairs = false;
    char* pmem = nullptr;
    int np1 = 0, np2 = 0;
};

namespace {

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

template <typename P>
DomDesc<P> make_desc(const lbps_lattice* lat) {
    DomDesc<P> d;
    d.g = lat->L.g;
    d.c = lat->c;
    d.k = lat->kc<P>();
    d.v[0] = lat->view<P>(0);
    d.v[1] = lat->view<P>(1);
    d.x = lat->xmem ? lat->copy_view<P>(lat->xmem) : lbps::View<P>{};
    d.bn = lat->bn();
    d.flag = lat->flag();
    d.tstep = lat->tstep();
    d.nb = lat->L.nb;
    d.cur = lat->cur;
    return d;
}

size_t desc_bytes(const lbps_batch* b) {
    return lbps::with_policy(b->storage, [](auto pol) { return sizeof(DomDesc<decltype(pol)>); });
}

// Work list of the interior kernel: every strip cut into chunks of `rows`
// rows; in a general geometry the rows of a strip without interior points
// (a hole, Geo::gap) are left out, splitting the chunk that spans them.  The
// list runs across a lattice's strips first, chunk row after chunk row, so
// warps that take consecutive tasks read neighbouring columns of the same
// rows (adjacent memory) at the same time.
std::vector<BulkTask> bulk_tasks(const lbps_batch* b, int rows) {
    std::vector<BulkTask> t;
    for (int d = 0; d < (int)b->lats.size(); ++d) {
        const lbps_lattice* lat = b->lats[d];
        const lbps::Geo& g = lat->L.g;
        for (int j0 = 0; j0 < g.ny; j0 += rows) {
            const int j1 = std::min(j0 + rows, g.ny);
            for (int xs = 0, s = 0; xs < g.nx; xs += lbps::kBatchStripCols, ++s) {
                const int ga = lat->gap.empty() ? 0 : lat->gap[2 * (size_t)s];
                const int gb = lat->gap.empty() ? 0 : lat->gap[2 * (size_t)s + 1];
                if (j0 < std::min(j1, ga)) t.push_back(BulkTask{d, xs, j0, std::min(j1, ga)});
                if (std::max(j0, gb) < j1) t.push_back(BulkTask{d, xs, std::max(j0, gb), j1});
            }
        }
    }
    return t;
}

// The Newmark pass of the boundary points as tasks of the persistent kernel:
// 32 consecutive entries of the boundary work list each, spread evenly
// through the strip tasks, so that warps gathering boundary data (latency
// bound) run among warps streaming the interior (bandwidth bound).
std::vector<BulkTask> with_newmark_tasks(const std::vector<BulkTask>& strips, int nbnd) {
    const size_t nn = (size_t)(nbnd + 31) / 32;
    std::vector<BulkTask> t;
    t.reserve(strips.size() + nn);
    size_t q = 0;
    for (size_t k = 0; k < nn; ++k) {
        // the k-th Newmark task goes before strip task k * strips / nn
        const size_t until = nn ? k * strips.size() / nn : 0;
        for (; q < until; ++q) t.push_back(strips[q]);
        const int b0 = (int)(32 * k);
        t.push_back(BulkTask{0, b0, -1, std::min(32, nbnd - b0)});
    }
    for (; q < strips.size(); ++q) t.push_back(strips[q]);
    return t;
}

// Largest work list for any rows >= 8: ceil(ny / 8) chunks per strip, one of
// them possibly split in two by the gap, and the Newmark tasks.
size_t max_bulk_tasks(const lbps_batch* b) {
    size_t n = 0, nbnd = 0;
    for (const lbps_lattice* lat : b->lats) {
        const lbps::Geo& g = lat->L.g;
        const size_t strips = (size_t)(g.nx + lbps::kBatchStripCols - 1) / lbps::kBatchStripCols;
        n += strips * ((size_t)(g.ny + 7) / 8 + 1);
        nbnd += (size_t)lat->L.nb;
    }
    return n + (nbnd + 31) / 32;
}

// The tasks of one stage of a pair of steps (two steps per sweep), as
// run_pair runs them on a single lattice: stage 1 the two-step strips
// (pair_kernel's 28 columns by 32 rows over the points at least 3 from every
// edge) and the frame strips on the points 1..3 from the edges; stage 2 the
// frame strips on the points 1..2 from the edges (frame_kernel's bands);
// both with the Newmark pass of every boundary point spread evenly among them.
std::vector<PairTask> pair_stage_tasks(const lbps_batch* b, int stage) {
    constexpr int kDeep = 3, kPairCols = 28, kRows = 32, kCols = lbps::kBatchStripCols;
    const int fw = stage == 1 ? 3 : 2;
    std::vector<PairTask> work;
    int nbnd = 0;
    for (int d = 0; d < (int)b->lats.size(); ++d) {
        const lbps::Geo& g = b->lats[d]->L.g;
        const int nx = g.nx, ny = g.ny;
        nbnd += b->lats[d]->L.nb;
        if (stage == 1)
            for (int j0 = kDeep; j0 < ny - kDeep; j0 += kRows)
                for (int xs = kDeep; xs < nx - kDeep; xs += kPairCols)
                    work.push_back(PairTask{d, lbps::kPairStrip, xs, j0, std::min(j0 + kRows, ny - kDeep), 0, 0, 0, 0});
        const int all = (nx + kCols - 1) / kCols;
        for (int q = 0; q < all; ++q) {   // top and bottom bands, fw rows each
            work.push_back(PairTask{d, lbps::kFrameStrip, q * kCols, 1, 1 + fw, 1, nx - 1, 1, 1 + fw});
            work.push_back(PairTask{d, lbps::kFrameStrip, q * kCols, ny - 1 - fw, ny - 1, 1, nx - 1, ny - 1 - fw,
                                    ny - 1});
        }
        const int jb = 1 + fw, je = ny - 1 - fw;   // left and right bands between them
        for (int j0 = jb; j0 < je; j0 += kRows) {
            const int j1 = std::min(j0 + kRows, je);
            for (int q = 1 / kCols; q <= fw / kCols; ++q)
                work.push_back(PairTask{d, lbps::kFrameStrip, q * kCols, j0, j1, 1, 1 + fw, jb, je});
            for (int q = (nx - 1 - fw) / kCols; q <= (nx - 2) / kCols; ++q)
                work.push_back(PairTask{d, lbps::kFrameStrip, q * kCols, j0, j1, nx - 1 - fw, nx - 1, jb, je});
        }
    }
    const size_t nn = (size_t)(nbnd + 31) / 32;
    std::vector<PairTask> t;
    t.reserve(work.size() + nn);
    size_t q = 0;
    for (size_t k = 0; k < nn; ++k) {
        const size_t until = k * work.size() / nn;
        for (; q < until; ++q) t.push_back(work[q]);
        const int b0 = (int)(32 * k);
        t.push_back(PairTask{0, lbps::kNewmarkTask, b0, 0, std::min(32, nbnd - b0), 0, 0, 0, 0});
    }
    for (; q < work.size(); ++q) t.push_back(work[q]);
    return t;
}

int fail(lbps_batch* b, cudaError_t e) {
    b->last_cuda = (int)e;
    return LBPS_ERR_CUDA;
}

// (Re)builds the bulk work list for b->rows and the descriptors, in a device
// block sized for the largest work list the tuner may ask for.
int upload(lbps_batch* b) {
    std::vector<BndTask> nt;
    for (int d = 0; d < (int)b->lats.size(); ++d)
        for (int q = 0; q < b->lats[d]->L.nb; ++q) nt.push_back(BndTask{d, q});
    std::vector<BulkTask> bt = with_newmark_tasks(bulk_tasks(b, b->rows), (int)nt.size());
    if (bt.size() > b->max_bulk) return LBPS_ERR_INVALID;  // cannot happen (see max_bulk_tasks)
    std::vector<char> host(b->off_bnd + nt.size() * sizeof(BndTask));
    size_t db = desc_bytes(b);
    for (int d = 0; d < (int)b->lats.size(); ++d) {
        lbps::with_policy(b->storage, [&](auto pol) {
            auto x = make_desc<decltype(pol)>(b->lats[d]);
            std::memcpy(host.data() + d * db, &x, db);
            return 0;
        });
        b->uploaded_cur[d] = b->lats[d]->cur;
        b->uploaded_gen[d] = b->lats[d]->gen;
    }
    std::memcpy(host.data() + b->off_bnd, nt.data(), nt.size() * sizeof(BndTask));
    cudaError_t e = cudaMemcpyAsync(b->mem, host.data(), host.size(), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->mem + b->off_bulk, bt.data(), bt.size() * sizeof(BulkTask), cudaMemcpyHostToDevice,
                            b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail(b, e);
    b->nbnd = (int)nt.size();
    b->nbulk = (int)bt.size();
    return LBPS_OK;
}

// One time step of every lattice: parity 0 reads v[cur], parity 1 v[cur ^ 1].
// Two launches: the persistent kernel runs the interior strips and, among
// them, the boundary Newmark tasks (those read copy A and write only the
// boundary points' u, du/dt of copy B, which no strip touches); the boundary
// reset follows (it reads the new u and overwrites populations the strips
// wrote).
cudaError_t launch_step(lbps_batch* b, int parity) {
    const BndTask* bt = reinterpret_cast<const BndTask*>(b->mem + b->off_bnd);
    const BulkTask* wt = reinterpret_cast<const BulkTask*>(b->mem + b->off_bulk);
    return lbps::with_policy(b->storage, [&](auto pol) {
        using P = decltype(pol);
        const DomDesc<P>* dd = reinterpret_cast<const DomDesc<P>*>(b->mem);
        unsigned* next = reinterpret_cast<unsigned*>(b->mem + b->off_next);
        cudaError_t e = lbps::launch_bulk_batch<P>(dd, wt, b->nbulk, bt, parity, b->variant, next, b->st);
        if (e == cudaSuccess) e = lbps::launch_boundary_batch<P>(dd, bt, b->nbnd, parity, 2, 3, b->st);
        return e;
    });
}

// Two steps of every lattice (two steps per sweep; parity as for launch_step,
// per pair): stage 1, the reset of the first step (v[a], x -> x), stage 2,
// the reset of the second (x, v[a ^ 1] -> v[a ^ 1]).
cudaError_t launch_pair_step(lbps_batch* b, int parity) {
    const BndTask* bt = reinterpret_cast<const BndTask*>(b->mem + b->off_bnd);
    const PairTask* p1 = reinterpret_cast<const PairTask*>(b->pmem);
    const PairTask* p2 = p1 + b->np1;
    return lbps::with_policy(b->storage, [&](auto pol) {
        using P = decltype(pol);
        const DomDesc<P>* dd = reinterpret_cast<const DomDesc<P>*>(b->mem);
        unsigned* next = reinterpret_cast<unsigned*>(b->mem + b->off_next) + 1;   // the two stages' counters
        cudaError_t e = cudaMemsetAsync(next, 0, 2 * sizeof(unsigned), b->st);
        if (e == cudaSuccess) e = lbps::launch_pair_batch<P>(dd, p1, b->np1, bt, parity, 1, next, b->st);
        if (e == cudaSuccess) e = lbps::launch_boundary_batch<P>(dd, bt, b->nbnd, parity, 2, 3, b->st, 1);
        if (e == cudaSuccess) e = lbps::launch_pair_batch<P>(dd, p2, b->np2, bt, parity, 2, next + 1, b->st);
        if (e == cudaSuccess) e = lbps::launch_boundary_batch<P>(dd, bt, b->nbnd, parity, 2, 3, b->st, 2);
        return e;
    });
}

void drop_graph(lbps_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->pair) cudaGraphExecDestroy(b->pair);
    b->graph = nullptr;
    b->pair = nullptr;
}

// Captures k steps as one graph: parities 0, 1, 0, 1, ... (k even, so the
// current copy is the same after it), or with `repeat` the parity-0 step k
// times (the autotuner's timing graph, which rewrites the same next state).
int capture(lbps_batch* b, int k, bool repeat, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail(b, e);
    cudaError_t e1 = cudaSuccess;
    for (int q = 0; q < k && e1 == cudaSuccess; ++q) e1 = launch_step(b, repeat ? 0 : q & 1);
    e = cudaStreamEndCapture(b->st, &g);
    if (e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return fail(b, e);
    }
    return LBPS_OK;
}

// Refreshes the descriptors if any lattice was stepped on its own (its
// current copy moved) or initialised again (its 16-bit scale may have
// changed) since the last upload.  The graph reads the descriptors from
// device memory, so it stays valid.
int refresh(lbps_batch* b) {
    for (size_t d = 0; d < b->lats.size(); ++d)
        if (b->lats[d]->cur != b->uploaded_cur[d] || b->lats[d]->gen != b->uploaded_gen[d]) return upload(b);
    return LBPS_OK;
}

}  // namespace

extern "C" {

int lbps_batch_create(lbps_lattice* const* lats, int32_t count, void* cuda_stream, lbps_batch** out) {
    if (!out || !lats || count < 1) return LBPS_ERR_INVALID;
    *out = nullptr;
    const int32_t storage = lats[0] ? lats[0]->p.storage : LBPS_STORAGE_F32;
    for (int32_t d = 0; d < count; ++d) {
        const lbps_lattice* l = lats[d];
        if (!l) return LBPS_ERR_INVALID;
        if (!l->initialised) return LBPS_ERR_STATE;
        if (l->p.storage != storage || l->p.sync_every != 0) return LBPS_ERR_INVALID;
        for (int32_t q = 0; q < d; ++q)
            if (lats[q] == l) return LBPS_ERR_INVALID;
    }
    lbps_batch* b = new (std::nothrow) lbps_batch();
    if (!b) return LBPS_ERR_OOM;
    b->lats.assign(lats, lats + count);
    b->uploaded_cur.assign(count, -1);
    b->uploaded_gen.assign(count, -1);
    b->storage = storage;
    if (cuda_stream) {
        b->st = reinterpret_cast<cudaStream_t>(cuda_stream);
    } else {
        // The legacy default stream cannot be captured; a blocking stream of
        // our own stays ordered with it.
        if (cudaStreamCreate(&b->st) != cudaSuccess) {
            delete b;
            return LBPS_ERR_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&b->order, cudaEventDisableTiming) != cudaSuccess) {
        lbps_batch_destroy(b);
        return LBPS_ERR_CUDA;
    }
    // Work lists: the bulk list sized for the longest any tile height gives.
    size_t max_bulk = max_bulk_tasks(b);
    b->max_bulk = max_bulk;
    size_t nbnd = 0;
    for (auto* l : b->lats) nbnd += (size_t)l->L.nb;
    b->off_bnd = align256((size_t)count * desc_bytes(b));
    b->off_bulk = align256(b->off_bnd + nbnd * sizeof(BndTask));
    b->off_next = align256(b->off_bulk + std::max<size_t>(max_bulk, 1) * sizeof(BulkTask));
    b->mem_bytes = b->off_next + 256;
    if (cudaMalloc(&b->mem, b->mem_bytes) != cudaSuccess) {
        cudaGetLastError();
        lbps_batch_destroy(b);
        return LBPS_ERR_OOM;
    }
    int rc = upload(b);
    if (rc != LBPS_OK) {
        lbps_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBPS_OK;
}

int lbps_batch_set_tuning(lbps_batch* b, int32_t variant, int32_t rows_per_warp) {
    if (!b || variant < 0 || variant >= lbps::kTuningVariants || rows_per_warp < 8 || rows_per_warp > 4096)
        return LBPS_ERR_INVALID;
    b->variant = variant;
    b->rows = rows_per_warp;
    drop_graph(b);
    return upload(b);
}

int lbps_batch_step(lbps_batch* b, int64_t n) {
    lbps::NvtxRange nvtx("lbps_batch_step");
    if (!b || n < 0) return LBPS_ERR_INVALID;
    if (n == 0) return LBPS_OK;
    // start after the work already queued on the lattices' own streams
    for (auto* l : b->lats) {
        if (l->st == b->st) continue;
        cudaError_t e = cudaEventRecord(b->order, l->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->order, 0);
        if (e != cudaSuccess) return fail(b, e);
    }
    int rc = refresh(b);
    if (rc != LBPS_OK) return rc;
    int flips = (int)(n & 1);   // how the current copy of every lattice moves
    int64_t q = 0;
    if (b->pairs) {
        // two steps per sweep: every pair writes the other copy (parity
        // alternating); an odd last step starts from the copy they leave
        const int64_t np = n / 2;
        for (int64_t k = 0; k < np; ++k) {
            cudaError_t e = launch_pair_step(b, (int)(k & 1));
            if (e != cudaSuccess) return fail(b, e);
        }
        q = 2 * np;
        flips = (int)((np & 1) ^ (n & 1));
        if (q < n) {
            cudaError_t e = launch_step(b, (int)(np & 1));
            if (e != cudaSuccess) return fail(b, e);
            q = n;
        }
    }
    // blocks of graph_k steps, then pairs, then a last single step
    if (b->graph_k > 2 && n - q >= b->graph_k) {
        if (!b->graph && (rc = capture(b, b->graph_k, false, &b->graph)) != LBPS_OK) return rc;
        for (; q + b->graph_k <= n; q += b->graph_k) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->st);
            if (e != cudaSuccess) return fail(b, e);
        }
    }
    if (n - q >= 2) {
        if (!b->pair && (rc = capture(b, 2, false, &b->pair)) != LBPS_OK) return rc;
        for (; q + 2 <= n; q += 2) {
            cudaError_t e = cudaGraphLaunch(b->pair, b->st);
            if (e != cudaSuccess) return fail(b, e);
        }
    }
    if (q < n) {
        cudaError_t e = launch_step(b, 0);
        if (e != cudaSuccess) return fail(b, e);
    }
    // later work on the lattices' own streams starts after these steps
    cudaError_t e = cudaEventRecord(b->order, b->st);
    for (auto* l : b->lats)
        if (e == cudaSuccess && l->st != b->st) e = cudaStreamWaitEvent(l->st, b->order, 0);
    if (e != cudaSuccess) return fail(b, e);
    for (auto* l : b->lats) {
        l->steps += n;
        l->cur ^= flips;
    }
    return LBPS_OK;
}

int lbps_batch_check(lbps_batch* b) {
    if (!b) return LBPS_ERR_INVALID;
    std::vector<unsigned> flags(b->lats.size(), 0);
    cudaError_t e = cudaSuccess;
    for (size_t d = 0; d < b->lats.size() && e == cudaSuccess; ++d)
        e = cudaMemcpyAsync(&flags[d], b->lats[d]->flag(), sizeof(unsigned), cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail(b, e);
    for (unsigned f : flags)
        if (f) return LBPS_ERR_NONFINITE;
    return LBPS_OK;
}

int lbps_batch_set_graph_steps(lbps_batch* b, int32_t k) {
    if (!b || k < 2 || k > 64 || (k & 1)) return LBPS_ERR_INVALID;
    b->graph_k = k;
    drop_graph(b);
    return LBPS_OK;
}

int lbps_batch_graph_steps(const lbps_batch* b) { return b ? b->graph_k : LBPS_ERR_INVALID; }

int lbps_batch_set_step_pairs(lbps_batch* b, int32_t on) {
    if (!b || (on != 0 && on != 1)) return LBPS_ERR_INVALID;
    if (b->st) cudaStreamSynchronize(b->st);
    if (b->pmem) cudaFree(b->pmem);
    b->pmem = nullptr;
    b->pairs = false;
    b->np1 = b->np2 = 0;
    if (!on) return LBPS_OK;
    for (lbps_lattice* l : b->lats) {
        const lbps::Geo& g = l->L.g;
        if (g.general || g.periodic_x || g.periodic_y || g.nx < 16 || g.ny < 16 || l->L.nb <= 0)
            return LBPS_ERR_INVALID;
    }
    for (lbps_lattice* l : b->lats) {   // the scratch copy of each lattice
        const int rc = lbps_set_step_pairs(l, 1);
        if (rc != LBPS_OK) return rc;
    }
    const std::vector<PairTask> t1 = pair_stage_tasks(b, 1), t2 = pair_stage_tasks(b, 2);
    if (cudaMalloc(&b->pmem, (t1.size() + t2.size()) * sizeof(PairTask)) != cudaSuccess) {
        cudaGetLastError();
        b->pmem = nullptr;
        return LBPS_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(b->pmem, t1.data(), t1.size() * sizeof(PairTask), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->pmem + t1.size() * sizeof(PairTask), t2.data(), t2.size() * sizeof(PairTask),
                            cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return fail(b, e);
    b->np1 = (int)t1.size();
    b->np2 = (int)t2.size();
    b->pairs = true;
    drop_graph(b);
    return upload(b);   // the descriptors with the scratch copies
}

int lbps_batch_step_pairs(const lbps_batch* b) { return b ? (int)b->pairs : LBPS_ERR_INVALID; }

int lbps_batch_tune(lbps_batch* b, int32_t repeats, int32_t* variant, int32_t* rows_per_warp, double* ms_per_step) {
    lbps::NvtxRange nvtx("lbps_batch_tune");
    if (!b || repeats < 1) return LBPS_ERR_INVALID;
    int rc = refresh(b);
    if (rc != LBPS_OK) return rc;
    const int rows_c[] = {8, 16, 32, 64, 128};
    const int var_c[] = {0, 1, 2, 4, 5, 6};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(b, cudaGetLastError());
    float best = -1.0f;
    int bv = b->variant, br = b->rows;
    for (int r : rows_c) {
        b->rows = r;
        drop_graph(b);
        rc = upload(b);
        if (rc != LBPS_OK) break;
        for (int v : var_c) {
            b->variant = v;
            // A step is a pure function of the copy it reads, so repeating the
            // parity-0 step rewrites the same next state: timing it leaves the
            // lattices where they were.
            cudaError_t e = launch_step(b, 0);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->st);
            for (int q = 0; q < repeats && e == cudaSuccess; ++q) e = launch_step(b, 0);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                rc = fail(b, e);
                break;
            }
            ms /= repeats;
            if (best < 0.0f || ms < best) {
                best = ms;
                bv = v;
                br = r;
            }
        }
        if (rc != LBPS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timed steps advanced the step counters (time of the boundary data):
    // put back the count of steps actually taken
    std::vector<unsigned long long> taken(b->lats.size());
    for (size_t d = 0; d < b->lats.size() && rc == LBPS_OK; ++d) {
        taken[d] = (unsigned long long)b->lats[d]->steps;
        cudaError_t e = cudaMemcpyAsync(b->lats[d]->tstep(), &taken[d], sizeof(taken[d]), cudaMemcpyHostToDevice,
                                        b->st);
        if (e != cudaSuccess) rc = fail(b, e);
    }
    if (rc == LBPS_OK) {
        cudaError_t e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) rc = fail(b, e);
    }
    if (rc != LBPS_OK) return rc;
    b->variant = bv;
    b->rows = br;
    drop_graph(b);
    rc = upload(b);
    if (rc != LBPS_OK) return rc;
    // Steps per graph for that launch shape: k repeats of the parity-0 step
    // captured as one graph, replayed `repeats` times (the same next state
    // again; the step counters are put back below).
    float best_g = -1.0f;
    int bk = b->graph_k;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return fail(b, cudaGetLastError());
    for (int k : {2, 4, 8, 16, 32}) {
        cudaGraphExec_t g = nullptr;
        rc = capture(b, k, true, &g);
        if (rc != LBPS_OK) break;
        cudaError_t e = cudaGraphLaunch(g, b->st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->st);
        for (int q = 0; q < repeats && e == cudaSuccess; ++q) e = cudaGraphLaunch(g, b->st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        cudaGraphExecDestroy(g);
        if (e != cudaSuccess) {
            rc = fail(b, e);
            break;
        }
        ms /= (float)(repeats * k);
        if (best_g < 0.0f || ms < 0.99f * best_g) {  // a longer graph must win by 1 %
            best_g = ms;
            bk = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (size_t d = 0; d < b->lats.size() && rc == LBPS_OK; ++d) {
        cudaError_t e = cudaMemcpyAsync(b->lats[d]->tstep(), &taken[d], sizeof(taken[d]), cudaMemcpyHostToDevice,
                                        b->st);
        if (e != cudaSuccess) rc = fail(b, e);
    }
    if (rc == LBPS_OK) {
        cudaError_t e = cudaStreamSynchronize(b->st);
        if (e != cudaSuccess) rc = fail(b, e);
    }
    if (rc != LBPS_OK) return rc;
    b->graph_k = bk;
    if (variant) *variant = bv;
    if (rows_per_warp) *rows_per_warp = br;
    if (ms_per_step) *ms_per_step = best_g;
    return LBPS_OK;
}

int lbps_batch_last_cuda_error(const lbps_batch* b) { return b ? b->last_cuda : 0; }

void lbps_batch_destroy(lbps_batch* b) {
    if (!b) return;
    if (b->st) cudaStreamSynchronize(b->st);
    drop_graph(b);
    if (b->mem) cudaFree(b->mem);
    if (b->pmem) cudaFree(b->pmem);
    if (b->order) cudaEventDestroy(b->order);
    if (b->own_stream) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"
