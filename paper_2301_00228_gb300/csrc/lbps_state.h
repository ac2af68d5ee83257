// Host-side state of a lattice, shared by the ABI translation units.
#pragma once

#include <cstdint>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbps.h"
#include "lbps_launch.h"

namespace lbps {

// NVTX range around an entry point (named lbps_* after it), so profilers can
// attribute GPU work to the call that enqueued it; costs nothing without a
// tool attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// The storage codes whose pair sums are held in 16 bits a value (PopNeq16,
// PopBfp13).
inline bool storage_is16(int32_t storage) {
    return storage == LBPS_STORAGE_BF16 || storage == LBPS_STORAGE_F16 || storage == LBPS_STORAGE_BFP13;
}

// Placement of everything in a lattice's device block.
struct Layout {
    Geo g;
    size_t f_bytes;     // population planes (layout of the storage policy), aligned
    size_t u_bytes;     // 4 FP64 planes, aligned
    size_t m_bytes;     // boundary mirror (g.mplane points, storage layout), aligned
    size_t s_bytes;     // stresses of the boundary cells (2 or 5 slots of 3 doubles per point), aligned
    size_t copy_bytes;
    size_t off_copy[2];
    size_t off_bn, off_type, off_gap, off_part, off_out, off_flag, off_staging;
    size_t staging_bytes;
    size_t total;
    int nb;
};

// Calls fn with a value of the storage policy type of an LBPS_STORAGE_* code.
template <typename Fn>
auto with_policy(int32_t storage, Fn&& fn) {
    switch (storage) {
    case LBPS_STORAGE_F64: return fn(PolF64{});
    case LBPS_STORAGE_BF16: return fn(PolBF16{});
    case LBPS_STORAGE_F16: return fn(PolF16{});
    case LBPS_STORAGE_BFP13: return fn(PolBfp13{});
    default: return fn(PolF32{});
    }
}

}  // namespace lbps

struct lbps_lattice {
    lbps_params p;
    lbps::Layout L;
    lbps::Consts c;
    lbps::KC<float> kf;
    lbps::KC<double> kd;
    double cd, cs, a_phi, a_psi, a0_psi;
    double bc_est = 0.0;  // boundary values' share of the 16-bit scale estimate
    int scale_exp = 0;    // 16-bit storage: Nx, Ny are stored times 2^scale_exp
    int64_t gen = 0;      // incremented by every init (batches re-read descriptors)
    uint64_t setup_hash = 0;  // parameters and boundary description (checked by lbps_state_load)
    std::vector<int> gap; // general geometry: rows without interior points per strip (Geo::gap, host copy)
    cudaStream_t st;
    // second stream for the boundary Newmark pass beside the interior kernel,
    // ordered by the fork/join events (null: the pass runs on st)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // time steps captured as CUDA graphs and replayed by lbps_step: [0] a
    // pair, [1] a block of graph_k (even) steps; one per starting copy
    // (captured on `cap`, a stream of the lattice's own, since the legacy
    // default stream cannot be captured); valid while graph_gen == gen
    cudaStream_t cap = nullptr;
    int graph_k = 32;   // 5-14 % faster than pairs below 1024^2, 3 % at 2048^2 (FP32)
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    int64_t graph_gen[2][2] = {{-1, -1}, {-1, -1}};
    int graph_cur[2][2] = {{0, 1}, {0, 1}};  // the current copy after a replay
    char* mem;
    bool owns;
    int cur;            // copy holding time t
    // two steps per sweep (lbps_set_step_pairs): the scratch state copy that
    // holds step n + 1 on the boundary and the points up to 3 from it
    // (cudaMalloc'd, copy_bytes), null when off
    char* xmem = nullptr;
    // pairs of steps of a lattice below lbps_solo_pairs_max points run as a
    // batch of this one lattice (lbps_step_async)
    lbps_batch* solo = nullptr;
    lbps::Tuning tuning;  // bulk-kernel launch shape
    int last_cuda = 0;    // cudaError_t of the last failing CUDA call
    int64_t steps;
    bool initialised;
    // per-kernel event timing (lbps_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<int> ev_kind;   // per recorded pair: 0 bulk, 1 boundary

    template <typename P>
    lbps::View<P> view(int q) const {
        return copy_view<P>(mem + L.off_copy[q]);
    }
    // A state copy laid out at base (the two copies of the block, or the
    // scratch copy of two-step sweeps).
    template <typename P>
    lbps::View<P> copy_view(char* base) const {
        lbps::View<P> v;
        v.f = reinterpret_cast<typename P::Base*>(base);
        v.u = reinterpret_cast<double*>(base + L.f_bytes);
        v.m = reinterpret_cast<typename P::Base*>(base + L.f_bytes + L.u_bytes);
        v.s = reinterpret_cast<double*>(base + L.f_bytes + L.u_bytes + L.m_bytes);
        return v;
    }
    double* u(int q) const { return reinterpret_cast<double*>(mem + L.off_copy[q] + L.f_bytes); }
    template <typename P>
    const lbps::KCof<P>& kc() const {
        if constexpr (std::is_same<typename P::V, double>::value)
            return kd;
        else
            return kf;
    }
    const lbps::BNode* bn() const { return reinterpret_cast<const lbps::BNode*>(mem + L.off_bn); }
    unsigned* flag() const { return reinterpret_cast<unsigned*>(mem + L.off_flag); }
    // device step counter (time of the boundary data), beside the flag
    unsigned long long* tstep() const { return reinterpret_cast<unsigned long long*>(mem + L.off_flag + 8); }
    double* partials() const { return reinterpret_cast<double*>(mem + L.off_part); }
    double* out4() const { return reinterpret_cast<double*>(mem + L.off_out); }
    double* staging() const { return reinterpret_cast<double*>(mem + L.off_staging); }
    bool neq16() const { return lbps::storage_is16(p.storage); }
};
