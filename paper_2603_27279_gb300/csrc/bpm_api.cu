// Host runtime and C ABI (include/bpm.h) of the bonded-particle rod library.
//
// The handle owns one device arena holding the SoA state, per-particle and
// per-bond constants, scratch for layout conversion and energies, plus the
// dipole work list and partial-sum buffer sized by the autotuner.
//
// A step runs three kernels: bond (+ Zeeman, damping, dipole orientation),
// dipole all-pairs partial sums, finish (reduce + velocity Verlet +
// Richardson).  bpm_step replays them from CUDA graphs of 16 steps, one step
// and the closing step, with no host round trip until the final read of the
// device error word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bpm_internal.h"

using namespace bpm;

namespace bpm {
int dipole_blocks_per_sm(bool mixed);
}

namespace {

thread_local std::string g_create_error;

// Autotuner cache: systems with the same work shape reuse the first choice,
// so every handle on a given system sums in the same order.  The value is
// (symmetric kernel?, its param).
using TuneKey = std::tuple<int, int, int64_t, int64_t, uint64_t>;
// the tuned plan; ovl_blocks: the dipole grid when the bond kernel runs beside
// it (ovl_bond: the bond grid then), 0 when it does not, -1 when not decided
struct TunedPlan {
    bool sym;
    int param;
    int ovl_blocks, ovl_bond;
};
std::map<TuneKey, TunedPlan> g_tune_cache;
std::mutex g_tune_mutex;

uint64_t hash_offsets(const std::vector<int64_t>& offs) {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : offs) {
        h ^= (uint64_t)v;
        h *= 1099511628211ull;
    }
    return h;
}

constexpr int kChunkSteps = 16;

}  // namespace

namespace bpm {
// error message of a failed call that has no handle (read by bpm_last_error(NULL))
void set_handleless_error(const std::string& msg) { g_create_error = msg; }
}  // namespace bpm

struct bpm_handle {
    int device = 0;
    int n_sm = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t n = 0, R = 0, n_bonds = 0;
    int dipole_mode = BPM_DIPOLE_OFF;
    bool mixed = false;  // BPM_MIXED: FP32 dipole pair terms
    bool ff = false;     // BPM_FF: float-float dipole pair terms
    double pairs = 0.0;  // ordered pairs per force evaluation

    Sys sys{};
    void* arena = nullptr;
    double* q_gauge = nullptr;  // SoA rest orientations (identity when none given)
    double* stage = nullptr;    // 4N staging for layout conversion
    double* energy_d = nullptr; // 5
    double* B_rod_d = nullptr;  // SoA [3][R]
    uint8_t* nslot_d = nullptr;
    int* counter_d = nullptr;
    int* pinned_err = nullptr;  // host pinned: err word
    double* pinned_e = nullptr; // host pinned: 5 energies

    // dipole work
    WorkItem* items_d = nullptr;
    int n_items = 0;
    size_t items_cap = 0;
    bool items_ragged = false;  // a work item's particle range ends inside a tile
    double* part_d = nullptr;
    int part_slots = 0;
    DipoleCfg cfg{};
    bool tuned = false;
    int tuned_split = 0;  // param of the plan in use (ordered: global j-chunks or per-rod chunk length)
    int plan_kind = BPM_PLAN_AUTO, plan_param = 0;

    bool forces_valid = false;

    // the bond kernel (FP64 pipe) beside the dipole kernel (FP32 pipe) on a
    // second stream, forked and joined by events
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    int overlap_mode = -1;   // bpm_set_overlap: -1 timed by the tuner, 0 off, 1 on
    bool overlap = false;    // in use
    int overlap_blocks = 0;  // dipole grid while overlapped
    int overlap_bond = 0;    // bond grid while overlapped (blocks that stay resident)

    cudaGraphExec_t g_chunk = nullptr, g_one = nullptr, g_last = nullptr;

    // contact between non-bonded particles
    bool has_contact = false;
    Contact ct{};

    // lattice Boltzmann fluid
    bool has_lbm = false;
    Lbm lbm{};
    void* lbm_mem = nullptr;
    double* lbm_scratch = nullptr;  // 4 * nodes doubles for bpm_lbm_fields
    int lbm_parity = 0;             // buffer holding the current distributions
    int lbm_phase = 0;              // DEM steps done in the current cycle
    int64_t lbm_nodes = 0;

    bool timing = false;
    double t_ms[5] = {0, 0, 0, 0, 0}, launches[5] = {0, 0, 0, 0, 0}, units[5] = {0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<int> ev_kind;
    std::vector<double> ev_units;

    std::string err;
    std::vector<int64_t> offs;  // host copy of the rod offsets (work lists)

    // adjoint record (bpm_adjoint_begin / bpm_adjoint_end)
    bool adj_recorded = false;
    int adj_steps = 0, adj_every = 0, adj_nck = 0;
    size_t adj_snap = 0;        // doubles per snapshot
    void* adj_arena = nullptr;
    size_t adj_bytes = 0;
    double *adj_ck = nullptr, *adj_seg = nullptr, *adj_work = nullptr;
    double *adj_wf = nullptr, *adj_wt = nullptr, *adj_wm = nullptr, *adj_out = nullptr;
    int* adj_dummy = nullptr;
    int64_t* adj_rod_off = nullptr;
    AdjBuf adj{};
};

namespace {

int fail(bpm_handle* h, int code, const std::string& msg) {
    if (h)
        h->err = msg;
    else
        g_create_error = msg;
    return code;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(h, BPM_ERR_CUDA, std::string("line ") + std::to_string(__LINE__) + ": " + \
                                             #call + ": " + cudaGetErrorString(e_));         \
    } while (0)

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void destroy_graphs(bpm_handle* h) {
    if (h->g_chunk) cudaGraphExecDestroy(h->g_chunk);
    if (h->g_one) cudaGraphExecDestroy(h->g_one);
    if (h->g_last) cudaGraphExecDestroy(h->g_last);
    h->g_chunk = h->g_one = h->g_last = nullptr;
}

// ---------------------------------------------------------------- timing
cudaEvent_t next_event(bpm_handle* h) {
    if (h->ev_used == h->ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev.push_back(e);
    }
    return h->ev[h->ev_used++];
}

template <class F>
cudaError_t timed_on(bpm_handle* h, cudaStream_t st, int kind, double units, F&& launch) {
    if (!h->timing) return launch();
    cudaEvent_t a = next_event(h), b = next_event(h);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    h->ev_kind.push_back(kind);
    h->ev_units.push_back(units);
    return e;
}
template <class F>
cudaError_t timed(bpm_handle* h, int kind, double units, F&& launch) {
    return timed_on(h, h->stream, kind, units, launch);
}

// Reads the recorded event pairs into the per-kind totals (synchronises the
// stream).  Called by bpm_get_timing, and by bpm_step / bpm_forces only when
// many pairs have piled up, so a timed call carries no extra host round trip.
constexpr size_t kTimingEventsMax = 4096;
int collect_timing(bpm_handle* h, bool force = true) {
    if (!h->timing || h->ev_used == 0) return BPM_OK;
    if (!force && h->ev_used < kTimingEventsMax) return BPM_OK;
    CK(cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < h->ev_kind.size(); ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]));
        h->t_ms[h->ev_kind[k]] += ms;
        h->launches[h->ev_kind[k]] += 1.0;
        h->units[h->ev_kind[k]] += h->ev_units[k];
    }
    h->ev_used = 0;
    h->ev_kind.clear();
    h->ev_units.clear();
    return BPM_OK;
}

// ---------------------------------------------------------------- dipole launch
// blocks: the persistent grid (the plan's, or fewer while the bond kernel
// runs beside it)
cudaError_t launch_dipole_any(bpm_handle* h, const Sys& s, int blocks, bool beside = false) {
    if (h->ff) {
        const cudaError_t e = launch_ff_encode(s, h->stream);
        if (e != cudaSuccess) return e;
        if (h->cfg.g == 0)
            return launch_dipole_symw_ff(s, h->items_d, h->n_items, h->counter_d, blocks, h->stream);
        return launch_dipole_sym_ff(s, h->items_d, h->n_items, h->counter_d, h->cfg.g, blocks, h->items_ragged,
                                    h->stream);
    }
    if (h->cfg.sym && h->cfg.g == 0)
        return h->mixed ? launch_dipole_symw_mixed(s, h->items_d, h->n_items, h->counter_d, blocks, h->stream)
                        : launch_dipole_symw_fp64(s, h->items_d, h->n_items, h->counter_d, blocks, h->stream);
    if (h->cfg.sym)
        return launch_dipole_sym(s, h->mixed, h->items_d, h->n_items, h->counter_d, h->cfg.g, blocks,
                                 h->items_ragged, h->stream);
    DipoleCfg c = h->cfg;
    c.blocks = blocks;
    return launch_dipole(s, h->mixed, h->items_d, h->n_items, h->counter_d, c, h->stream, beside);
}
cudaError_t launch_dipole_any(bpm_handle* h, const Sys& s) { return launch_dipole_any(h, s, h->cfg.blocks); }

// m for all particles, then the dipole kernel (main stream, `blocks` blocks)
// and the bond kernel (side stream) at the same time, joined on the main
// stream.  The two write disjoint buffers (partial slots; f and tau).
template <class Orient, class Dipole, class Bond>
cudaError_t launch_overlapped(bpm_handle* h, Orient&& orient, Dipole&& dipole, Bond&& bond) {
    cudaError_t e = orient();
    if (e != cudaSuccess) return e;
    if ((e = cudaEventRecord(h->fork_ev, h->stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(h->side, h->fork_ev, 0)) != cudaSuccess) return e;
    if ((e = dipole()) != cudaSuccess) return e;
    if ((e = bond()) != cudaSuccess) return e;
    if ((e = cudaEventRecord(h->join_ev, h->side)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(h->stream, h->join_ev, 0);
}

// particles per tile of the symmetric kernel of this handle's precision
int sym_tile(const bpm_handle* h) { return h->ff ? dipole_ff_tile() : dipole_sym_tile(h->mixed); }
int sym_blocks_per_sm(const bpm_handle* h, int g) {
    return h->ff ? dipole_ff_blocks_per_sm(g) : dipole_sym_blocks_per_sm(h->mixed, g);
}
int prec_of(const bpm_handle* h) { return h->ff ? BPM_FF : (h->mixed ? BPM_MIXED : BPM_FP64); }
// particles per tile pair item of symmetric plan g (g = 0: 32-particle tiles,
// one warp per pair)
// particles per tile of the warp-tile plan (g = 0): 32, or 64 for the packed
// FP32 pairs, whose lanes hold two i and meet two j per instruction
int64_t symw_tile(const bpm_handle* h) { return h->mixed ? 64 : 32; }
int64_t sym_span(const bpm_handle* h, int g) { return g == 0 ? symw_tile(h) : (int64_t)g * sym_tile(h); }
int symw_blocks_per_sm(const bpm_handle* h) {
    if (h->ff) return dipole_symw_ff_blocks_per_sm();
    return h->mixed ? dipole_symw_mixed_blocks_per_sm() : dipole_symw_blocks_per_sm();
}

// ---------------------------------------------------------------- dipole work list
// A tuning candidate: the symmetric kernel with g tiles per supertile, or the
// ordered-pair kernel with a j-split (global: number of j-chunks; per rod:
// j-chunk length).
struct Cand {
    bool sym;
    int param;
};

// Balances the end of a symmetric supertile pass over one interacting set.
// Its items are mostly whole supertile pairs of equal cost, handed out
// largest first from the atomic queue. With W of them over B persistent
// blocks, some blocks end one whole item after the others unless W is a
// multiple of B. Blocks on one SM share its pipes, so the others there
// speed up when one runs dry, and the loss is small: cutting the tail
// gained 0.2 % (FP64) to 0.5 % (float-float) on the helix and the cilia
// array. B of the whole off-diagonal items, taken round-robin over I, are
// cut into two halves along j. The halves go to the end of the queue with
// the diagonal items, which cost about the same. The first half keeps the item's
// slots. The second half writes its i side to a slot of its own past the T
// partner slots (each particle of I then has T + e(I) slots) and its j side
// to slot I, as before. Only the kernels that skip j subtiles past a ragged
// end take such halves (FP64 and float-float), and only while every
// particle keeps at most 255 slots.
void split_tail(const bpm_handle* h, int g, int64_t st, std::vector<WorkItem>& items, std::vector<uint8_t>& nslot,
                int& max_slots) {
    const int64_t T = max_slots;
    if (T < 2 || st % 64 != 0) return;
    const int64_t blocks = (int64_t)h->n_sm * std::max(1, sym_blocks_per_sm(h, g));
    std::vector<std::vector<size_t>> by_i((size_t)T);
    size_t whole = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        const WorkItem& w = items[k];
        if (!w.pad1 && w.ni == st && w.nj == st) {
            by_i[(size_t)w.pad0].push_back(k);
            ++whole;
        }
    }
    const int64_t S = std::min<int64_t>(blocks, (int64_t)whole);
    std::vector<size_t> chosen;
    for (size_t round = 0; (int64_t)chosen.size() < S; ++round) {
        bool any = false;
        for (int64_t I = 0; I < T && (int64_t)chosen.size() < S; ++I)
            if (round < by_i[(size_t)I].size()) {
                chosen.push_back(by_i[(size_t)I][round]);
                any = true;
            }
        if (!any) break;
    }
    std::vector<int> extra((size_t)T, 0);
    for (size_t k : chosen) ++extra[(size_t)items[k].pad0];
    const int emax = *std::max_element(extra.begin(), extra.end());
    if (T + emax > 255) return;
    std::fill(extra.begin(), extra.end(), 0);
    const int32_t half = (int32_t)(st / 2);
    for (size_t k : chosen) {
        WorkItem& w = items[k];
        WorkItem h2 = w;
        w.nj = half;
        h2.j0 = w.j0 + half;
        h2.nj = (int32_t)st - half;
        h2.slot = (int32_t)(T + extra[(size_t)w.pad0]++);
        items.push_back(h2);
    }
    for (int64_t I = 0; I < T; ++I)
        for (int64_t i = I * st; i < std::min<int64_t>((I + 1) * st, h->n); ++i)
            nslot[(size_t)i] = (uint8_t)(T + extra[(size_t)I]);
    max_slots = (int)(T + emax);
}

void build_items(const bpm_handle* h, const std::vector<int64_t>& offs, Cand cand,
                 std::vector<WorkItem>& items, std::vector<uint8_t>& nslot, int& max_slots) {
    items.clear();
    nslot.assign((size_t)h->n, 0);
    max_slots = 0;
    if (cand.sym) {
        const int64_t st = sym_span(h, cand.param);
        auto add_range = [&](int64_t b, int64_t L) {
            const int64_t T = (L + st - 1) / st;
            for (int64_t I = 0; I < T; ++I)
                for (int64_t J = I; J < T; ++J) {
                    WorkItem w{};
                    w.i0 = (int32_t)(b + I * st);
                    w.ni = (int32_t)std::min<int64_t>(st, b + L - w.i0);
                    w.j0 = (int32_t)(b + J * st);
                    w.nj = (int32_t)std::min<int64_t>(st, b + L - w.j0);
                    w.slot = (int32_t)J;  // i side: partner supertile J
                    w.pad0 = (int32_t)I;  // j side: partner supertile I
                    w.pad1 = I == J ? 1 : 0;
                    items.push_back(w);
                }
            for (int64_t i = b; i < b + L; ++i) nslot[(size_t)i] = (uint8_t)std::min<int64_t>(T, 255);
            max_slots = std::max<int>(max_slots, (int)T);
        };
        if (h->dipole_mode == BPM_DIPOLE_GLOBAL) {
            if (h->n >= 2) add_range(0, h->n);
            if (cand.param > 0 && !h->mixed) split_tail(h, cand.param, st, items, nslot, max_slots);
        } else if (h->dipole_mode == BPM_DIPOLE_PER_ROD) {
            for (int64_t r = 0; r < h->R; ++r) {
                const int64_t b = offs[(size_t)r], L = offs[(size_t)r + 1] - b;
                if (L >= 2) add_range(b, L);
            }
        }
        std::stable_sort(items.begin(), items.end(), [](const WorkItem& a, const WorkItem& b) {
            const int64_t ca = (int64_t)a.ni * a.nj / (a.pad1 ? 2 : 1), cb = (int64_t)b.ni * b.nj / (b.pad1 ? 2 : 1);
            return ca > cb;
        });
        return;
    }
    const int split = cand.param;
    const int ti = dipole_tile_i(h->mixed, h->cfg);
    auto add_range = [&](int64_t b, int64_t L, int S) {
        const int64_t chunk = (L + S - 1) / S;
        int used = 0;
        for (int s = 0; s < S; ++s) {
            const int64_t j0 = b + s * chunk;
            const int64_t nj = std::min<int64_t>(chunk, b + L - j0);
            if (nj <= 0) break;
            ++used;
            for (int64_t i0 = b; i0 < b + L; i0 += ti) {
                WorkItem w{};
                w.i0 = (int32_t)i0;
                w.ni = (int32_t)std::min<int64_t>(ti, b + L - i0);
                w.j0 = (int32_t)j0;
                w.nj = (int32_t)nj;
                w.slot = s;
                items.push_back(w);
            }
        }
        for (int64_t i = b; i < b + L; ++i) nslot[(size_t)i] = (uint8_t)used;
        max_slots = std::max(max_slots, used);
    };
    if (h->dipole_mode == BPM_DIPOLE_GLOBAL) {
        if (h->n >= 2) add_range(0, h->n, split);
    } else if (h->dipole_mode == BPM_DIPOLE_PER_ROD) {
        for (int64_t r = 0; r < h->R; ++r) {
            const int64_t b = offs[(size_t)r], L = offs[(size_t)r + 1] - b;
            if (L < 2) continue;
            const int S = (int)std::min<int64_t>(255, (L + split - 1) / split);
            add_range(b, L, S);
        }
    }
    // largest items first: the atomic queue then hands them out in LPT order
    std::stable_sort(items.begin(), items.end(), [](const WorkItem& a, const WorkItem& b) {
        return (int64_t)a.ni * a.nj > (int64_t)b.ni * b.nj;
    });
}

int upload_items(bpm_handle* h, const std::vector<WorkItem>& items, const std::vector<uint8_t>& nslot,
                 int max_slots) {
    if (items.size() > h->items_cap) {
        if (h->items_d) cudaFree(h->items_d);
        h->items_d = nullptr;
        CK(cudaMalloc(&h->items_d, items.size() * sizeof(WorkItem)));
        h->items_cap = items.size();
    }
    if (!items.empty())
        CK(cudaMemcpyAsync(h->items_d, items.data(), items.size() * sizeof(WorkItem),
                           cudaMemcpyHostToDevice, h->stream));
    h->n_items = (int)items.size();
    const int tile = sym_tile(h);
    h->items_ragged = false;
    for (const WorkItem& w : items)
        if (w.ni % tile != 0 || w.nj % tile != 0) {
            h->items_ragged = true;
            break;
        }
    // grown when needed; shrunk when a plan needs less than half (the tuner
    // may have tried a plan with many slots)
    if (max_slots > h->part_slots || (max_slots > 0 && 2 * max_slots < h->part_slots)) {
        if (h->part_d) cudaFree(h->part_d);
        h->part_d = nullptr;
        CK(cudaMalloc(&h->part_d, (size_t)max_slots * 7 * (size_t)h->n * sizeof(double)));
        h->part_slots = max_slots;
    }
    if (h->n > 0)
        CK(cudaMemcpyAsync(h->nslot_d, nslot.data(), (size_t)h->n, cudaMemcpyHostToDevice, h->stream));
    h->sys.part = h->part_d;
    h->sys.S = max_slots;
    CK(cudaStreamSynchronize(h->stream));  // host vectors go out of scope
    return BPM_OK;
}

// a pair of timing events, destroyed on every return path of the tuners
struct TimingEvents {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&a);
        return e != cudaSuccess ? e : cudaEventCreate(&b);
    }
    ~TimingEvents() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// Whether db blocks of d and bb blocks of b are resident on one SM at once
// (registers, shared memory with the per-block reserve, threads, blocks).
bool fit_side_by_side(int device, const BlockRes& d, int db, const BlockRes& b, int bb) {
    if (d.threads == 0 || b.threads == 0) return false;
    int regs = 0, smem = 0, threads = 0, blocks = 0, reserve = 0;
    if (cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&threads, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&blocks, cudaDevAttrMaxBlocksPerMultiprocessor, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (int64_t)d.regs * d.threads * db + (int64_t)b.regs * b.threads * bb <= regs &&
           (int64_t)(d.smem + reserve) * db + (int64_t)(b.smem + reserve) * bb <= smem &&
           d.threads * db + b.threads * bb <= threads && db + bb <= blocks;
}

// Whether the bond kernel runs beside the dipole kernel (*dipole_blocks > 0)
// and with which grids.  The bond kernel keeps the FP64 pipe busy and the
// FP32-pair dipole kernels the FP32 pipe, so on BPM_MIXED and BPM_FF handles
// the two can share the SMs.  Both grids are sized to stay resident side by
// side (registers, shared memory, threads: fit_side_by_side): the dipole
// kernel one or two blocks per SM below its occupancy, the bond kernel up to
// three blocks per SM looping over its particle groups, so the outcome does
// not depend on which kernel the hardware dispatches first.  In automatic
// mode the sequential form and the first form that fits are timed (bond and
// dipole, from m to the join) and the faster is kept (the overlapped one by a
// margin of 3 %); *best_ms is its time
// over two launches (sequential or overlapped), or negative when nothing was
// timed.  Systems with contact or a fluid, forced plans, FP64 handles and
// dipole passes too long to time take the sequential form unless
// bpm_set_overlap(h, 1) asks for it.
int decide_overlap(bpm_handle* h, bool forced_plan, int cached, int cached_bond, int* dipole_blocks,
                   int* bond_blocks, bool* timed_here, float* best_ms = nullptr) {
    *dipole_blocks = 0;
    *bond_blocks = 0;
    *timed_here = false;
    if (best_ms) *best_ms = -1.f;
    const bool eligible = h->side && !h->has_contact && !h->has_lbm && h->n_items > 0 && h->n_bonds > 0;
    if (!eligible || h->overlap_mode == 0) return BPM_OK;
    const int bps = std::max(1, h->cfg.blocks / std::max(1, h->n_sm));
    const BlockRes dres = h->ff ? dipole_ff_block_res(h->cfg.sym ? h->cfg.g : 0)
                                : dipole_block_res(h->mixed, h->cfg.sym != 0, h->cfg.g, true);
    const BlockRes bres = bond_side_block_res(h->sys.hist != nullptr);
    // (dipole, bond) blocks per SM that fit side by side: for each dipole
    // count the two largest bond counts
    std::vector<std::pair<int, int>> fits;
    for (int db = std::max(1, bps - 1); db >= std::max(1, bps - 2); --db) {
        int added = 0;
        for (int bb = 3; bb >= 1 && added < 2; --bb)
            if (fit_side_by_side(h->device, dres, db, bres, bb)) {
                fits.push_back({db, bb});
                ++added;
            }
    }
    if (h->overlap_mode == 1) {
        // forced: the largest dipole grid with the most bond blocks that fit
        // (or one block each below the dipole kernel's occupancy)
        const std::pair<int, int> f = fits.empty() ? std::pair<int, int>{std::max(1, bps - 1), 1} : fits[0];
        *dipole_blocks = h->n_sm * f.first;
        *bond_blocks = h->n_sm * f.second;
        return BPM_OK;
    }
    if (forced_plan || !(h->mixed || h->ff) || h->pairs > (h->mixed ? 3e10 : 1e10)) return BPM_OK;
    if (cached >= 0) {
        *dipole_blocks = cached;
        *bond_blocks = cached_bond;
        return BPM_OK;
    }
    Sys s = h->sys;
    s.count_step = 0;
    auto run = [&](int db, int bb) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(h->counter_d, 0, sizeof(int), h->stream);
        if (e != cudaSuccess) return e;
        if (db == 0) {
            e = launch_bond(s, false, h->mixed, false, 0, h->stream);
            return e != cudaSuccess ? e : launch_dipole_any(h, s);
        }
        return launch_overlapped(
            h, [&] { return launch_orient(s, h->mixed, h->stream); },
            [&] { return launch_dipole_any(h, s, db, true); },
            [&] { return launch_bond(s, false, false, true, bb, h->side); });
    };
    // Only the first fitting form (most dipole blocks, then most bond blocks)
    // is timed against the sequential one. A form that leaves room on an SM
    // lets the block scheduler place the two grids unevenly, depending on
    // which kernel it dispatches first, and that order differs between these
    // eager trials and the captured graphs: on the batched rods such a form
    // (2 dipole and 1 bond block per SM) timed 1 % faster here than the form
    // that fills the register file (2 and 2) and ran 7 % slower in the steps.
    std::vector<std::pair<int, int>> forms = {{0, 0}};
    if (!fits.empty()) forms.push_back({h->n_sm * fits[0].first, h->n_sm * fits[0].second});
    TimingEvents ev;
    CK(ev.create());
    cudaEvent_t a = ev.a, b = ev.b;
    float best = 1e30f;
    for (const auto& f : forms) {
        float sum = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(a, h->stream));
            CK(run(f.first, f.second));
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (rep > 0) sum += ms;
        }
        // the overlapped form must beat the sequential one by 3 %: these
        // eager trials favour it slightly against the captured steps (the
        // helix with FP32 pairs: 1 % faster here, 1 % slower in the steps)
        const bool seq = f.first == 0;
        if (seq ? sum < best : sum < 0.97f * best) {
            best = sum;
            *dipole_blocks = f.first;
            *bond_blocks = f.second;
        }
    }
    CK(cudaMemsetAsync(h->counter_d, 0, sizeof(int), h->stream));
    *timed_here = true;
    if (best_ms) *best_ms = best;
    return BPM_OK;
}

// Picks the dipole work decomposition by timing candidates (a project
// autotuner): the symmetric kernel with 1, 2, 3, 4, 5, 6 or 8 tiles per supertile
// (FP64 path) and the ordered-pair kernel with a few j-splits.  Runs once, at
// the first force evaluation, after the bond kernel has written m; the choice
// is cached per work shape.  Systems whose dipole pass is too expensive to
// time several times take the occupancy heuristic.
int tune_dipole(bpm_handle* h, const std::vector<int64_t>& offs) {
    if (h->tuned || h->dipole_mode == BPM_DIPOLE_OFF) return BPM_OK;
    const int bps = std::max(1, dipole_blocks_per_sm(h->mixed));
    const int ordered_blocks = h->n_sm * bps;
    // largest rod (or the system) in particles, for the partial-buffer bound
    int64_t Lmax = h->n;
    if (h->dipole_mode == BPM_DIPOLE_PER_ROD) {
        Lmax = 0;
        for (int64_t r = 0; r < h->R; ++r) Lmax = std::max(Lmax, offs[(size_t)r + 1] - offs[(size_t)r]);
    }
    const double part_cap = 2.0e9;  // bytes of partial sums allowed
    std::vector<Cand> cands;
    {
        // warp tiles, one warp per pair: one partial per partner tile, for
        // systems whose supertile pairs are too few to fill the GPU, and rods
        // whose lengths leave supertiles ragged; the slot traffic is charged
        // to it below
        const int64_t T = (Lmax + symw_tile(h) - 1) / symw_tile(h);
        if (T <= 255 && (double)T * 7.0 * 8.0 * (double)h->n <= part_cap && symw_blocks_per_sm(h) > 0)
            cands.push_back({true, 0});
    }
    {
        // a kernel's shared memory (and so its blocks per SM) grows with g:
        // the sizes in between are tried as well
        for (int g : {1, 2, 3, 4, 5, 6, 8}) {
            const int64_t st = (int64_t)g * sym_tile(h);
            const int64_t T = (Lmax + st - 1) / st;
            if (T > 255 || (double)T * 7.0 * 8.0 * (double)h->n > part_cap) continue;
            if (sym_blocks_per_sm(h, g) < 1) continue;
            cands.push_back({true, g});
        }
    }
    const int ti = dipole_tile_i(h->mixed, h->cfg);
    if (h->ff) {
        // the float-float path has the symmetric kernel only
    } else if (h->dipole_mode == BPM_DIPOLE_GLOBAL) {
        const int64_t tiles = (h->n + ti - 1) / ti;
        const int target = 2 * ordered_blocks;
        const int heur = (int)std::min<int64_t>(64, std::max<int64_t>(1, (target + tiles - 1) / tiles));
        bool any = false;
        for (int s : {1, 2, 4, 8, 16, 32, 64})
            if (s >= heur / 4 && s <= std::max(heur * 2, 1) && s <= h->n) {
                cands.push_back({false, s});
                any = true;
            }
        if (!any) cands.push_back({false, heur});
    } else {
        for (int c : {256, 512, 1024, 2048, 1 << 30}) cands.push_back({false, c});
    }
    // the pair count bounds what timing may cost: then the first symmetric
    // candidate with enough items, else the heuristic ordered split
    if (cands.empty()) return fail(h, BPM_ERR_ARG, "no runnable dipole plan for this system");
    if (h->pairs > (h->mixed ? 3e10 : (h->ff ? 1e10 : 1e9))) {
        Cand pick = cands.back();
        for (const Cand& c : cands)
            if (!c.sym) { pick = c; break; }
        for (const Cand& c : cands)
            if (c.sym) { pick = c; break; }
        cands = {pick};
    }
    std::vector<WorkItem> items;
    std::vector<uint8_t> nslot;
    int max_slots = 0;
    Cand best = cands[0];
    const TuneKey key{h->dipole_mode, prec_of(h), h->n, h->R, hash_offsets(offs)};
    const bool forced = h->plan_kind != BPM_PLAN_AUTO;
    int cached_ovl = -1, cached_bond = 0;
    if (forced) {
        best = Cand{h->plan_kind == BPM_PLAN_SYMMETRIC, h->plan_param};
        cands = {best};
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = Cand{it->second.sym, it->second.param};
            cached_ovl = it->second.ovl_blocks;
            cached_bond = it->second.ovl_bond;
            cands = {best};
        }
    }
    auto configure = [&](Cand c) {
        h->cfg.sym = c.sym ? 1 : 0;
        h->cfg.g = c.sym ? c.param : 0;
        h->cfg.blocks = !c.sym ? ordered_blocks
                                : h->n_sm * std::max(1, c.param == 0 ? symw_blocks_per_sm(h) : sym_blocks_per_sm(h, c.param));
    };
    std::vector<std::pair<float, Cand>> costs;  // candidates' times alone, with the slot reads
    std::vector<double> slot_ms;                 // their slot reads (two launches)
    if (cands.size() > 1) {
        TimingEvents ev;
        CK(ev.create());
        cudaEvent_t a = ev.a, b = ev.b;
        float best_ms = 1e30f;
        for (Cand c : cands) {
            build_items(h, offs, c, items, nslot, max_slots);
            int rc = upload_items(h, items, nslot, max_slots);
            if (rc) return rc;
            configure(c);
            float ms_sum = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                CK(cudaMemsetAsync(h->counter_d, 0, sizeof(int), h->stream));
                CK(cudaEventRecord(a, h->stream));
                CK(launch_dipole_any(h, h->sys));
                CK(cudaEventRecord(b, h->stream));
                CK(cudaEventSynchronize(b));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, a, b));
                if (rep > 0) ms_sum += ms;
            }
            // the partial slots the kernel wrote are read back by the finish
            // kernel (past four slots by the slot reduction, which writes and
            // the finish kernel reads one slot more): that traffic, at about
            // 6.5 TB/s, is charged to the candidate as well
            double slot_entries = 0.0;
            for (uint8_t k : nslot) slot_entries += k;
            if (max_slots > 4) slot_entries += 2.0 * (double)h->n;
            const double read_ms = slot_entries * 7.0 * 8.0 / 6.5e12 * 1e3;
            ms_sum += 2.0f * (float)read_ms;  // two timed launches
            costs.push_back({ms_sum, c});
            slot_ms.push_back(2.0 * read_ms);
            if (ms_sum < best_ms) {
                best_ms = ms_sum;
                best = c;
            }
        }
        CK(cudaMemsetAsync(h->counter_d, 0, sizeof(int), h->stream));
    }
    int ovl = 0, ovl_bond = 0;
    bool ovl_timed = false, joint = false;
    if (costs.size() > 1) {
        // Where the bond kernel can run beside the dipole kernel, the two
        // fastest candidates are timed again with the bond kernel, in their
        // sequential and overlapped forms, and the fastest plan and form are
        // kept: a plan that is slower alone can be faster beside the bond
        // kernel (its blocks fit better, or it writes fewer partial slots).
        std::vector<size_t> order(costs.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return costs[x].first < costs[y].first; });
        float best_total = 1e30f;
        for (size_t r = 0; r < std::min<size_t>(2, order.size()); ++r) {
            const Cand c = costs[order[r]].second;
            build_items(h, offs, c, items, nslot, max_slots);
            int rc = upload_items(h, items, nslot, max_slots);
            if (rc) return rc;
            configure(c);
            int db = 0, bb = 0;
            bool th = false;
            float fm = -1.f;
            rc = decide_overlap(h, forced, -1, 0, &db, &bb, &th, &fm);
            if (rc) return rc;
            if (fm < 0.f) break;  // no overlap form for this handle
            const float total = fm + (float)slot_ms[order[r]];
            if (total < best_total) {
                best_total = total;
                best = c;
                ovl = db;
                ovl_bond = bb;
                ovl_timed = th;
                joint = true;
            }
        }
    }
    build_items(h, offs, best, items, nslot, max_slots);
    int rc = upload_items(h, items, nslot, max_slots);
    if (rc) return rc;
    configure(best);
    if (!joint) rc = decide_overlap(h, forced, cached_ovl, cached_bond, &ovl, &ovl_bond, &ovl_timed);
    if (rc) return rc;
    h->overlap = ovl > 0;
    h->overlap_blocks = ovl;
    h->overlap_bond = ovl_bond;
    if (!forced) {
        // the overlap choice is kept only where it was timed
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = ovl_timed ? TunedPlan{best.sym, best.param, ovl, ovl_bond}
                                      : TunedPlan{best.sym, best.param, cached_ovl, cached_bond};
    }
    h->tuned = true;
    h->tuned_split = best.param;
    return BPM_OK;
}

// ---------------------------------------------------------------- launches
int launch_forces_sys_impl(bpm_handle* h, Sys s, int mode, bool energy, bool count_step);

int launch_forces_sys(bpm_handle* h, Sys s, int mode, bool energy, bool count_step) {
    int rc = launch_forces_sys_impl(h, s, mode, energy, count_step);
    if (rc)
        h->err += " (dipole plan sym=" + std::to_string(h->cfg.sym) + " g=" + std::to_string(h->cfg.g) +
                  " blocks=" + std::to_string(h->cfg.blocks) + " items=" + std::to_string(h->n_items) +
                  " slots=" + std::to_string(s.S) + " mode=" + std::to_string(mode) + ")";
    return rc;
}

int launch_forces_sys_impl(bpm_handle* h, Sys s, int mode, bool energy, bool count_step) {
    s.count_step = count_step ? 1 : 0;
    const bool dip = h->dipole_mode != BPM_DIPOLE_OFF && h->n_items > 0;
    if (dip && h->overlap && !energy && !h->has_contact && !h->has_lbm) {
        CK(launch_overlapped(
            h, [&] { return timed(h, 2, (double)h->n, [&] { return launch_orient(s, h->mixed, h->stream); }); },
            [&] { return timed(h, 1, h->pairs, [&] { return launch_dipole_any(h, s, h->overlap_blocks, true); }); },
            [&] {
                return timed_on(h, h->side, 0, (double)h->n_bonds,
                                [&] { return launch_bond(s, false, false, true, h->overlap_bond, h->side); });
            }));
    } else {
        CK(timed(h, 0, (double)h->n_bonds,
                 [&] { return launch_bond(s, energy, h->mixed && dip, false, 0, h->stream); }));
        if (h->has_contact) CK(timed(h, 3, (double)h->n, [&] { return launch_contact(s, h->ct, h->stream); }));
        if (h->has_lbm) CK(timed(h, 2, (double)h->n, [&] { return launch_ibm_penalty(s, h->lbm, h->stream); }));
        if (dip) CK(timed(h, 1, h->pairs, [&] { return launch_dipole_any(h, s); }));
    }
    // many partial slots: sum them on the whole GPU first
    s.slots_reduced = 0;
    if (dip && s.S > 4) {
        CK(timed(h, 2, (double)h->n, [&] { return launch_reduce_slots(s, h->stream); }));
        s.slots_reduced = 1;
    }
    CK(timed(h, 2, (double)h->n, [&] { return launch_finish(s, dip, mode, energy, h->counter_d, h->stream); }));
    return BPM_OK;
}

int launch_forces_like(bpm_handle* h, int mode, bool energy, bool count_step) {
    return launch_forces_sys(h, h->sys, mode, energy, count_step);
}

int capture(bpm_handle* h, int steps, int last_mode, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = BPM_OK;
    for (int k = 0; k < steps && rc == BPM_OK; ++k)
        rc = launch_forces_like(h, k + 1 == steps ? last_mode : FINISH_CONTINUE, false, true);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(h, BPM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, BPM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return BPM_OK;
}

int ensure_graphs(bpm_handle* h) {
    if (h->g_chunk) return BPM_OK;
    int rc = capture(h, kChunkSteps, FINISH_CONTINUE, &h->g_chunk);
    if (!rc) rc = capture(h, 1, FINISH_CONTINUE, &h->g_one);
    if (!rc) rc = capture(h, 1, FINISH_HALF_KICK, &h->g_last);
    if (rc) destroy_graphs(h);
    return rc;
}

int compute_forces(bpm_handle* h, bool energy) {
    if (h->n == 0) return BPM_OK;
    if (!h->tuned && h->dipole_mode != BPM_DIPOLE_OFF) {
        // m must exist before the tuner times the dipole kernel
        Sys s = h->sys;
        s.count_step = 0;
        CK(launch_bond(s, false, h->mixed, false, 0, h->stream));
        if (h->ff) CK(launch_ff_encode(s, h->stream));
        int rc = tune_dipole(h, h->offs);
        if (rc) return rc;
    }
    int rc = launch_forces_like(h, FINISH_FORCES, energy, false);
    if (rc) return rc;
    h->forces_valid = true;
    return BPM_OK;
}

// host or device source -> SoA device destination
int upload_aos(bpm_handle* h, const double* src, double* dst_soa, int nc) {
    if (h->n == 0) return BPM_OK;
    const double* dsrc = src;
    if (!is_device_ptr(src)) {
        CK(cudaMemcpyAsync(h->stage, src, (size_t)h->n * nc * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        dsrc = h->stage;
    }
    CK(launch_aos_to_soa(dsrc, dst_soa, h->n, nc, h->stream));
    return BPM_OK;
}

// SoA device source -> host or device AoS destination
int download_aos(bpm_handle* h, const double* src_soa, double* dst, int nc, bool* need_sync) {
    if (h->n == 0) return BPM_OK;
    if (is_device_ptr(dst)) {
        CK(launch_soa_to_aos(src_soa, dst, h->n, nc, h->stream));
        return BPM_OK;
    }
    CK(launch_soa_to_aos(src_soa, h->stage, h->n, nc, h->stream));
    CK(cudaMemcpyAsync(dst, h->stage, (size_t)h->n * nc * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // stage is reused by the next copy
    if (need_sync) *need_sync = false;
    return BPM_OK;
}

}  // namespace

// ---------------------------------------------------------------- contact capacity
namespace {
// queue a copy of the contact overflow flag (read after the caller's sync)
int queue_overflow_read(bpm_handle* h) {
    if (!h->has_contact) return BPM_OK;
    CK(cudaMemcpyAsync(h->pinned_err + 2, h->ct.overflow, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->ct.overflow, 0, sizeof(int), h->stream));
    return BPM_OK;
}
int check_overflow(bpm_handle* h) {
    if (!h->has_contact || h->pinned_err[2] == 0) return BPM_OK;
    h->pinned_err[2] = 0;
    h->forces_valid = false;
    return fail(h, BPM_ERR_CAPACITY,
                "a particle had more than " + std::to_string(h->ct.cap) +
                    " contacts; raise bpm_contact.max_contacts (the extra contacts kept no history)");
}
}  // namespace

// ---------------------------------------------------------------- adjoint
namespace {

// a Sys whose state lives in a snapshot block [x 3N | q 4N | v 3N | w 3N | t]
Sys snap_view(bpm_handle* h, double* block) {
    Sys s = h->sys;
    const int64_t n = h->n;
    s.x = block;
    s.q = block + 3 * n;
    s.v = block + 7 * n;
    s.w = block + 10 * n;
    s.tdev = block + 13 * n;
    s.f = h->adj_wf;
    s.t = h->adj_wt;
    s.m = h->adj_wm;
    s.err = h->adj_dummy;
    s.step_counter = h->adj_dummy + 1;
    s.count_step = 0;
    return s;
}

int snapshot_handle(bpm_handle* h, double* dst) {
    const size_t n = (size_t)h->n;
    CK(cudaMemcpyAsync(dst, h->sys.x, 3 * n * 8, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(dst + 3 * n, h->sys.q, 4 * n * 8, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(dst + 7 * n, h->sys.v, 3 * n * 8, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(dst + 10 * n, h->sys.w, 3 * n * 8, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(dst + 13 * n, h->sys.tdev, 8, cudaMemcpyDeviceToDevice, h->stream));
    return BPM_OK;
}

int adj_alloc(bpm_handle* h, int steps, int every) {
    const size_t n = (size_t)h->n;
    const size_t snap = (13 * n + 1 + 31) & ~size_t(31);
    const int nck = (steps + every - 1) / every;
    // dipole VJP: the symmetric form (one slot per 32-particle tile) for
    // all-pairs dipoles of one interacting set while its slots take at
    // most 512 MB; otherwise j-chunks, enough blocks to fill the GPU
    const int64_t tiles = ((int64_t)n + 31) / 32;
    const bool one_set = h->dipole_mode == BPM_DIPOLE_GLOBAL || (h->dipole_mode == BPM_DIPOLE_PER_ROD && h->R == 1);
    const bool sym = one_set && h->plan_kind != BPM_PLAN_ORDERED && 48.0 * (double)n * (double)tiles <= 512.0 * (1 << 20);
    const int64_t blocks = ((int64_t)n + 127) / 128;
    const int S = sym ? (int)tiles
                      : (int)std::max<int64_t>(1, std::min<int64_t>(32, (4 * (int64_t)h->n_sm + blocks - 1) / blocks));
    // BPM_FF handles with the symmetric form: float-float VJP inputs
    const size_t ff_floats = (h->ff && sym) ? (size_t)adj_ff_comp() * n : 0;
    const size_t doubles = snap * ((size_t)nck + (size_t)every + 2) + 9 * n + 52 * n + 6 * (size_t)S * n + 8 +
                           (ff_floats + 1) / 2 + 32;
    const size_t bytes = doubles * 8 + 256 + 8 * ((size_t)h->R + 1);
    if (bytes > h->adj_bytes) {
        if (h->adj_arena) cudaFree(h->adj_arena);
        h->adj_arena = nullptr;
        h->adj_bytes = 0;
        CK(cudaMalloc(&h->adj_arena, bytes));
        h->adj_bytes = bytes;
    }
    double* p = (double*)h->adj_arena;
    h->adj_snap = snap;
    h->adj_nck = nck;
    h->adj_ck = p;
    p += snap * nck;
    h->adj_seg = p;
    p += snap * ((size_t)every + 1);
    h->adj_work = p;
    p += snap;
    h->adj_wf = p;
    p += 3 * n;
    h->adj_wt = p;
    p += 3 * n;
    h->adj_wm = p;
    p += 3 * n;
    AdjBuf& A = h->adj;
    double** fields3[] = {&A.ax, &A.av, &A.aw, &A.aF, &A.aT, &A.amb, &A.aB, &A.m, &A.mu, &A.dx, &A.dm};
    for (double** f : fields3) {
        *f = p;
        p += 3 * n;
    }
    A.aq = p;
    p += 4 * n;
    A.bL = p;
    p += 7 * n;
    A.bR = p;
    p += 7 * n;
    A.dpart = p;
    A.S = S;
    A.sym = sym ? 1 : 0;
    p += 6 * (size_t)S * n;
    h->adj_out = p;
    p += 8;
    h->adj_dummy = (int*)p;
    p += 32;
    h->adj_rod_off = (int64_t*)p;
    p += (size_t)h->R + 1;
    A.ffbuf = ff_floats ? (float*)(((uintptr_t)p + 255) & ~(uintptr_t)255) : nullptr;
    CK(cudaMemcpyAsync(h->adj_rod_off, h->offs.data(), 8 * h->offs.size(), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return BPM_OK;
}

}  // namespace

// ============================================================== C ABI
extern "C" {

const char* bpm_version(void) { return "bpm-gb300 0.1 (sm_103a)"; }

const char* bpm_last_error(const bpm_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

namespace {

// Device pointer of the current device (or managed memory)?
bool is_device_ptr_of(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
}

// Shared by bpm_create (st == NULL: the handle owns its state arrays) and
// bpm_create_device (st: the state arrays are the caller's, used in place).
int create_impl(const bpm_desc* d_in, const bpm_device_state* st, bpm_handle** out) {
    bpm_handle* h = nullptr;
    if (!out) return fail(nullptr, BPM_ERR_ARG, "bpm_create: out is NULL");
    *out = nullptr;
    if (!d_in) return fail(nullptr, BPM_ERR_ARG, "bpm_create: desc is NULL");
    // a device-state handle: read the caller's initial state to the host once
    // and run the ordinary preparation on it (rest orientations the identity)
    bpm_desc dd = *d_in;
    std::vector<double> st_x, st_q, st_v, st_w, st_qr;
    if (st) {
        const int64_t Nd = d_in->n_particles;
        if (d_in->x || d_in->q || d_in->v || d_in->omega)
            return fail(nullptr, BPM_ERR_ARG, "bpm_create_device: x, q, v and omega of the description must be NULL");
        if (d_in->q_rest)
            return fail(nullptr, BPM_ERR_ARG, "bpm_create_device: q_rest must be NULL (rest orientations are the identity)");
        if (Nd < 0 || Nd > (int64_t)INT32_MAX / 2) return fail(nullptr, BPM_ERR_ARG, "bad n_particles");
        if (Nd > 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, BPM_ERR_CUDA, "no CUDA device");
            const double* ptrs[6] = {st->x, st->q, st->v, st->omega, st->f, st->tau};
            const char* names[6] = {"x", "q", "v", "omega", "f", "tau"};
            for (int k = 0; k < 6; ++k)
                if (!ptrs[k] || !is_device_ptr_of(ptrs[k], dev))
                    return fail(nullptr, BPM_ERR_ARG, std::string("bpm_create_device: st->") + names[k] +
                                                          " is not device memory of the current device");
            const size_t nd = (size_t)Nd;
            std::vector<double> soa(4 * nd);
            auto fetch = [&](const double* src, int nc, std::vector<double>& dst) {
                if (cudaMemcpy(soa.data(), src, (size_t)nc * nd * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
                dst.resize((size_t)nc * nd);
                for (size_t i = 0; i < nd; ++i)
                    for (int c = 0; c < nc; ++c) dst[(size_t)nc * i + c] = soa[(size_t)c * nd + i];
                return true;
            };
            if (!fetch(st->x, 3, st_x) || !fetch(st->q, 4, st_q) || !fetch(st->v, 3, st_v) || !fetch(st->omega, 3, st_w))
                return fail(nullptr, BPM_ERR_CUDA, "bpm_create_device: reading the initial state failed");
            st_qr.assign(4 * nd, 0.0);
            for (size_t i = 0; i < nd; ++i) st_qr[4 * i] = 1.0;
            dd.x = st_x.data();
            dd.q = st_q.data();
            dd.v = st_v.data();
            dd.omega = st_w.data();
            dd.q_rest = st_qr.data();
        }
    }
    const bpm_desc* d = &dd;
    const bool ext = st != nullptr && d->n_particles > 0;
    const int64_t N = d->n_particles, R = d->n_rods;
    if (N < 0 || R < 0) return fail(nullptr, BPM_ERR_ARG, "negative n_particles or n_rods");
    if (N > (int64_t)INT32_MAX / 2) return fail(nullptr, BPM_ERR_ARG, "n_particles exceeds 2^30");
    if (N > 0 && (R < 1 || !d->rod_offset)) return fail(nullptr, BPM_ERR_ARG, "rods: need n_rods >= 1 and rod_offset");
    if (N > 0 && (!d->x || !d->q || !d->mass || !d->radius))
        return fail(nullptr, BPM_ERR_ARG, "x, q, mass and radius are required");
    if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(nullptr, BPM_ERR_ARG, "dt must be > 0");
    if (!(d->damping >= 0.0)) return fail(nullptr, BPM_ERR_ARG, "damping must be >= 0");
    if (d->dipole_mode < 0 || d->dipole_mode > 2) return fail(nullptr, BPM_ERR_ARG, "bad dipole_mode");
    if (d->precision != BPM_FP64 && d->precision != BPM_MIXED && d->precision != BPM_FF)
        return fail(nullptr, BPM_ERR_ARG, "bad precision");
    const bpm_contact* cd = N > 0 ? d->contact : nullptr;
    int ct_cap = 0;
    if (cd) {
        if (!(cd->E > 0.0) || !std::isfinite(cd->E) || !(cd->nu > -1.0 && cd->nu < 0.5) || !(cd->mu >= 0.0) ||
            !std::isfinite(cd->mu) || !(cd->gamma_n >= 0.0) || !std::isfinite(cd->gamma_n) ||
            !(cd->gamma_t >= 0.0) || !std::isfinite(cd->gamma_t) || cd->exclude < 0)
            return fail(nullptr, BPM_ERR_ARG, "contact: need E > 0, -1 < nu < 0.5, mu, gamma_n, gamma_t >= 0, exclude >= 0");
        ct_cap = cd->max_contacts == 0 ? 16 : cd->max_contacts;
        if (ct_cap < 1 || ct_cap > 64) return fail(nullptr, BPM_ERR_ARG, "contact: max_contacts must be in 1..64");
        if (N > (int64_t)1 << 21) return fail(nullptr, BPM_ERR_ARG, "contact: at most 2^21 particles");
    }
    const bpm_lbm* ld = N > 0 ? d->lbm : nullptr;
    if (ld) {
        if (ld->nx < 1 || ld->ny < 1 || ld->nz < 1 || ld->n_sub < 1)
            return fail(nullptr, BPM_ERR_ARG, "lbm: need nx, ny, nz, n_sub >= 1");
        if (!(ld->tau > 0.5) || !std::isfinite(ld->tau)) return fail(nullptr, BPM_ERR_ARG, "lbm: tau must be > 0.5");
        if (std::fabs(d->dt * ld->n_sub - 1.0) > 1e-9)
            return fail(nullptr, BPM_ERR_ARG, "lbm: lattice units need dt * n_sub = 1");
        for (int k = 0; k < 3; ++k)
            if (!std::isfinite(ld->body_force[k])) return fail(nullptr, BPM_ERR_ARG, "lbm: body_force must be finite");
    }
    bool bond_damped = false;
    if (d->bond_damping && N > 0) {
        for (int64_t k = 0; k < 4 * R; ++k) {
            const double g = d->bond_damping[k];
            if (!(g >= 0.0) || !std::isfinite(g)) return fail(nullptr, BPM_ERR_ARG, "bond_damping must be finite and >= 0");
            if (g != 0.0) bond_damped = true;
        }
    }
    std::vector<int64_t> offs;
    if (N > 0) {
        offs.assign(d->rod_offset, d->rod_offset + R + 1);
        if (offs[0] != 0 || offs[(size_t)R] != N) return fail(nullptr, BPM_ERR_ARG, "rod_offset must run from 0 to N");
        for (int64_t r = 0; r < R; ++r)
            if (offs[(size_t)r + 1] < offs[(size_t)r]) return fail(nullptr, BPM_ERR_ARG, "rod_offset not non-decreasing");
    }
    // ---- host-side preparation (SoA)
    const size_t n = (size_t)N;
    std::vector<double> x(3 * n), q(4 * n), v(3 * n, 0.0), w(3 * n, 0.0), mb(3 * n, 0.0), mass(n), inertia(n);
    std::vector<double> inv_mass(n), inv_inertia(n);
    std::vector<double> qg(4 * n), bond(8 * n, 0.0);
    std::vector<uint8_t> flags(n, 0);
    std::vector<int32_t> rod_of(n, 0);
    int64_t n_bonds = 0;
    for (int64_t r = 0; r < R && N > 0; ++r)
        for (int64_t k = offs[(size_t)r]; k < offs[(size_t)r + 1]; ++k) rod_of[(size_t)k] = (int32_t)r;
    for (size_t i = 0; i < n; ++i) {
        const double* qi = d->q + 4 * i;
        const double qn = std::sqrt(qi[0] * qi[0] + qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]);
        if (!(qn > 0.0) || !std::isfinite(qn)) return fail(nullptr, BPM_ERR_ARG, "zero or non-finite quaternion");
        const double* qr = d->q_rest ? d->q_rest + 4 * i : qi;
        const double rn = std::sqrt(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        if (!(rn > 0.0) || !std::isfinite(rn)) return fail(nullptr, BPM_ERR_ARG, "zero or non-finite rest quaternion");
        // current orientation relative to rest: q' = q q_rest*, and the body
        // dipole expressed in that gauge: m~' = q_rest m~ q_rest*
        double a[4] = {qi[0] / qn, qi[1] / qn, qi[2] / qn, qi[3] / qn};
        double g[4] = {qr[0] / rn, qr[1] / rn, qr[2] / rn, qr[3] / rn};
        double c[4] = {g[0], -g[1], -g[2], -g[3]};
        double p[4] = {a[0] * c[0] - a[1] * c[1] - a[2] * c[2] - a[3] * c[3],
                       a[0] * c[1] + a[1] * c[0] + a[2] * c[3] - a[3] * c[2],
                       a[0] * c[2] - a[1] * c[3] + a[2] * c[0] + a[3] * c[1],
                       a[0] * c[3] + a[1] * c[2] - a[2] * c[1] + a[3] * c[0]};
        const double pn = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
        for (int k = 0; k < 4; ++k) {
            q[k * n + i] = p[k] / pn;
            qg[k * n + i] = g[k];
        }
        double m0[3] = {0, 0, 0};
        if (d->m_body) {
            m0[0] = d->m_body[3 * i];
            m0[1] = d->m_body[3 * i + 1];
            m0[2] = d->m_body[3 * i + 2];
        }
        // rotate by g: v + w t + u x t, t = 2 u x v
        double u[3] = {g[1], g[2], g[3]};
        double t[3] = {2 * (u[1] * m0[2] - u[2] * m0[1]), 2 * (u[2] * m0[0] - u[0] * m0[2]),
                       2 * (u[0] * m0[1] - u[1] * m0[0])};
        double rm[3] = {m0[0] + g[0] * t[0] + (u[1] * t[2] - u[2] * t[1]),
                        m0[1] + g[0] * t[1] + (u[2] * t[0] - u[0] * t[2]),
                        m0[2] + g[0] * t[2] + (u[0] * t[1] - u[1] * t[0])};
        for (int k = 0; k < 3; ++k) {
            x[k * n + i] = d->x[3 * i + k];
            mb[k * n + i] = rm[k];
            if (d->v) v[k * n + i] = d->v[3 * i + k];
            if (d->omega) w[k * n + i] = d->omega[3 * i + k];
        }
        if (!(d->mass[i] > 0.0) || !(d->radius[i] > 0.0)) return fail(nullptr, BPM_ERR_ARG, "mass and radius must be > 0");
        mass[i] = d->mass[i];
        inertia[i] = 0.4 * d->mass[i] * d->radius[i] * d->radius[i];
        inv_mass[i] = 1.0 / mass[i];
        inv_inertia[i] = 1.0 / inertia[i];
        if (d->clamped && d->clamped[i]) {
            flags[i] |= F_CLAMPED;
            for (int k = 0; k < 3; ++k) v[k * n + i] = w[k * n + i] = 0.0;
        }
    }
    // bonds: rest vector in the global frame of the rest state, spring constants
    if (N > 0) {
        const double* xr = d->x_rest ? d->x_rest : d->x;
        for (int64_t r = 0; r < R; ++r) {
            if (offs[(size_t)r + 1] - offs[(size_t)r] < 2) continue;
            if (!d->E || !d->nu || !d->d) return fail(nullptr, BPM_ERR_ARG, "E, nu and d are required for rods with bonds");
            const double E = d->E[r], nu = d->nu[r], dd = d->d[r];
            if (!(E > 0.0) || !(dd > 0.0) || !(nu > -1.0)) return fail(nullptr, BPM_ERR_ARG, "bad material");
            const double G = E / (2.0 * (1.0 + nu));
            const double A = M_PI * dd * dd / 4.0, I = M_PI * std::pow(dd, 4) / 64.0, J = M_PI * std::pow(dd, 4) / 32.0;
            for (int64_t k = offs[(size_t)r]; k + 1 < offs[(size_t)r + 1]; ++k) {
                const size_t kk = (size_t)k;
                double ri[3] = {xr[3 * kk + 3] - xr[3 * kk], xr[3 * kk + 4] - xr[3 * kk + 1], xr[3 * kk + 5] - xr[3 * kk + 2]};
                const double L = std::sqrt(ri[0] * ri[0] + ri[1] * ri[1] + ri[2] * ri[2]);
                if (!(L > 0.0)) return fail(nullptr, BPM_ERR_SINGULAR, "zero-length rest bond at particle " + std::to_string(k));
                const double vals[8] = {ri[0] / L, ri[1] / L, ri[2] / L, L, E * A / L, 12.0 * E * I / (L * L * L), G * J / L, E * I / L};
                for (int c = 0; c < 8; ++c) bond[c * n + kk] = vals[c];
                flags[kk] |= F_BOND_RIGHT;
                ++n_bonds;
            }
        }
    }

    // ---- device
    h = new (std::nothrow) bpm_handle();
    if (!h) return fail(nullptr, BPM_ERR_ARG, "out of host memory");
    h->offs = offs;
    auto bail = [&](int code) {
        g_create_error = h->err;
        bpm_destroy(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        h->err = "no CUDA device";
        return bail(BPM_ERR_CUDA);
    }
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device);
    h->n = N;
    h->R = R;
    h->n_bonds = n_bonds;
    h->dipole_mode = d->dipole_mode;
    h->mixed = d->precision == BPM_MIXED;
    h->ff = d->precision == BPM_FF;
    if (d->stream) {
        h->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            h->err = "stream creation failed";
            return bail(BPM_ERR_CUDA);
        }
        h->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess) {
        h->err = "side stream creation failed";
        return bail(BPM_ERR_CUDA);
    }
    {
        double pairs = 0.0;
        if (d->dipole_mode == BPM_DIPOLE_GLOBAL)
            pairs = (double)N * (double)(N > 0 ? N - 1 : 0);
        else if (d->dipole_mode == BPM_DIPOLE_PER_ROD)
            for (int64_t r = 0; r < R; ++r) {
                const double L = (double)(offs[(size_t)r + 1] - offs[(size_t)r]);
                pairs += L * (L - 1.0);
            }
        h->pairs = pairs;
    }
    // arena
    const size_t nn = std::max<size_t>(n, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    // state and forces: in the arena, or the caller's arrays (device handle)
    const size_t o_x = ext ? 0 : take(3 * nn * 8), o_q = ext ? 0 : take(4 * nn * 8),
                 o_v = ext ? 0 : take(3 * nn * 8), o_w = ext ? 0 : take(3 * nn * 8);
    const size_t o_f = ext ? 0 : take(3 * nn * 8), o_t = ext ? 0 : take(3 * nn * 8), o_m = take(3 * nn * 8),
                 o_mb = take(3 * nn * 8);
    const size_t o_mass = take(nn * 8), o_in = take(nn * 8), o_bond = take(8 * nn * 8), o_qg = take(4 * nn * 8);
    const size_t o_imass = take(nn * 8), o_iin = take(nn * 8);
    const size_t o_stage = take(4 * nn * 8), o_e = take(5 * nn * 8), o_en = take(5 * 8), o_t0 = take(8);
    const size_t o_err = take(4), o_sc = take(4), o_ctr = take(4), o_flags = take(nn), o_rod = take(nn * 4),
                 o_ns = take(nn), o_brod = take(3 * std::max<size_t>((size_t)R, 1) * 8);
    size_t o_bg = 0, o_hist = 0, o_gen = 0;
    if (bond_damped) {
        o_bg = take(4 * (size_t)R * 8);
        o_hist = take(6 * nn * 8);
    }
    if (bond_damped || cd) o_gen = take(4);
    // contact: cell list and two levels of tangential histories
    uint32_t ct_H = 64;
    while (cd && ct_H < 2 * nn) ct_H <<= 1;
    size_t o_ck = 0, o_cc = 0, o_cs = 0, o_co = 0, o_cb = 0, o_cp = 0, o_cx = 0, o_cn = 0, o_cv = 0, o_cf = 0,
           o_cr = 0, o_cxf = 0, o_crf = 0;
    if (cd) {
        o_ck = take(nn * 4);
        o_cc = take((size_t)ct_H * 4);
        o_cs = take(((size_t)ct_H + 1) * 4);
        o_co = take(nn * 4);
        o_cb = take((size_t)(contact_scan_blocks(ct_H) + 1) * 4);
        o_cp = take(2 * (size_t)ct_cap * nn * 4);
        o_cx = take(6 * (size_t)ct_cap * nn * 8);
        o_cn = take(2 * nn * 4);
        o_cv = take(2 * 4);
        o_cf = take(4);
        o_cr = take(nn * 8);
        o_cxf = take(3 * nn * 4);
        o_crf = take(nn * 4);
    }
    size_t o_xh = 0, o_xl = 0, o_mf = 0, o_xq = 0, o_mq = 0;
    if (h->mixed) {
        o_xh = take(3 * nn * 4);
        o_xl = take(3 * nn * 4);
        o_mf = take(3 * nn * 4);
    }
    if (h->ff) {
        o_xq = take(9 * nn * 4);
        o_mq = take(6 * nn * 4);
    }
    if (cudaMalloc(&h->arena, off) != cudaSuccess) {
        cudaGetLastError();
        h->err = "device allocation of " + std::to_string(off) + " bytes failed";
        return bail(BPM_ERR_CUDA);
    }
    char* A = (char*)h->arena;
    Sys& s = h->sys;
    s.n = N;
    if (ext) {
        s.x = st->x;
        s.q = st->q;
        s.v = st->v;
        s.w = st->omega;
        s.f = st->f;
        s.t = st->tau;
    } else {
        s.x = (double*)(A + o_x);
        s.q = (double*)(A + o_q);
        s.v = (double*)(A + o_v);
        s.w = (double*)(A + o_w);
        s.f = (double*)(A + o_f);
        s.t = (double*)(A + o_t);
    }
    s.m = (double*)(A + o_m);
    s.m_body = (const double*)(A + o_mb);
    s.mass = (const double*)(A + o_mass);
    s.inertia = (const double*)(A + o_in);
    s.inv_mass = (const double*)(A + o_imass);
    s.inv_inertia = (const double*)(A + o_iin);
    s.bond = (const double*)(A + o_bond);
    h->q_gauge = (double*)(A + o_qg);
    h->stage = (double*)(A + o_stage);
    s.e_part = (double*)(A + o_e);
    h->energy_d = (double*)(A + o_en);
    s.tdev = (double*)(A + o_t0);
    s.err = (int*)(A + o_err);
    s.step_counter = (int*)(A + o_sc);
    h->counter_d = (int*)(A + o_ctr);
    s.flags = (const uint8_t*)(A + o_flags);
    s.rod_of = (const int32_t*)(A + o_rod);
    h->nslot_d = (uint8_t*)(A + o_ns);
    s.nslot = h->nslot_d;
    h->B_rod_d = (double*)(A + o_brod);
    if (h->mixed) {
        s.xh = (float*)(A + o_xh);
        s.xl = (float*)(A + o_xl);
        s.mf = (float*)(A + o_mf);
    }
    if (h->ff) {
        s.xq = (float*)(A + o_xq);
        s.mq = (float*)(A + o_mq);
        // finest position digit 2^q with 2^(q+66) >= 4 max|x| + 64: room for
        // the system to spread to four times its initial extent
        double xmax = 0.0;
        for (int64_t i = 0; i < 3 * N; ++i)
            if (std::isfinite(d->x[i])) xmax = std::max(xmax, std::fabs(d->x[i]));
        int k = 0;
        while (std::ldexp(1.0, k) < 4.0 * xmax + 64.0) ++k;
        s.q_exp = k - 66;
    }
    if (bond_damped || cd) {
        s.hist_gen = (int*)(A + o_gen);
        if (cudaMemset(s.hist_gen, 0, 4) != cudaSuccess) {
            h->err = "history setup failed";
            return bail(BPM_ERR_CUDA);
        }
    }
    if (bond_damped) {
        std::vector<double> bg(4 * (size_t)R);
        for (int64_t r = 0; r < R; ++r)
            for (int k = 0; k < 4; ++k) bg[(size_t)k * R + r] = d->bond_damping[4 * r + k];
        s.bond_g = (const double*)(A + o_bg);
        s.hist = (double*)(A + o_hist);
        // all-ones bytes are a NaN: no measures recorded yet
        if (cudaMemcpy((void*)s.bond_g, bg.data(), bg.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(s.hist, 0xFF, 6 * nn * 8) != cudaSuccess) {
            h->err = "upload of bond_damping failed";
            return bail(BPM_ERR_CUDA);
        }
    }
    if (cd) {
        Contact& c = h->ct;
        h->has_contact = true;
        const double G = cd->E / (2.0 * (1.0 + cd->nu));
        c.E_star = cd->E / (2.0 * (1.0 - cd->nu * cd->nu));
        c.G_star = G / (2.0 * (2.0 - cd->nu));
        c.mu = cd->mu;
        c.gamma_n = cd->gamma_n;
        c.gamma_t = cd->gamma_t;
        double rmax = 0.0;
        for (size_t i = 0; i < n; ++i) rmax = std::max(rmax, d->radius[i]);
        c.inv_cell = 1.0 / (2.0 * rmax);
        c.exclude = cd->exclude;
        c.cap = ct_cap;
        c.H = ct_H;
        c.key = (int*)(A + o_ck);
        c.count = (int*)(A + o_cc);
        c.start = (int*)(A + o_cs);
        c.order = (int*)(A + o_co);
        c.block_sums = (int*)(A + o_cb);
        c.partner = (int*)(A + o_cp);
        c.xi = (double*)(A + o_cx);
        c.ncont = (int*)(A + o_cn);
        s.ct_valid = (int*)(A + o_cv);
        c.overflow = (int*)(A + o_cf);
        c.radius = (const double*)(A + o_cr);
        c.xf = (float*)(A + o_cxf);
        c.radf = (const float*)(A + o_crf);
        std::vector<float> rf(n);
        for (size_t i = 0; i < n; ++i) rf[i] = (float)d->radius[i];
        if (cudaMemcpy((void*)c.radius, d->radius, n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy((void*)c.radf, rf.data(), n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(c.count, 0, (size_t)ct_H * 4) != cudaSuccess || cudaMemset(s.ct_valid, 0, 8) != cudaSuccess ||
            cudaMemset(c.overflow, 0, 4) != cudaSuccess || cudaMemset(c.ncont, 0, 2 * nn * 4) != cudaSuccess) {
            h->err = "contact setup failed";
            return bail(BPM_ERR_CUDA);
        }
    }
    if (ld) {
        Lbm& L = h->lbm;
        h->has_lbm = true;
        L.nx = ld->nx;
        L.ny = ld->ny;
        L.nz = ld->nz;
        L.n_sub = ld->n_sub;
        L.tau = ld->tau;
        L.omega = 1.0 / ld->tau;
        L.gfac = 1.0 - 0.5 / ld->tau;
        L.omegaf = (float)L.omega;
        L.gfacf = (float)L.gfac;
        for (int k = 0; k < 3; ++k) {
            L.body[k] = ld->body_force[k];
            L.bodyf[k] = (float)ld->body_force[k];
        }
        L.fp32 = h->mixed ? 1 : 0;
        L.ff = h->ff ? 1 : 0;
        auto split2 = [](double v, float* out) {
            out[0] = (float)v;
            out[1] = (float)(v - (double)out[0]);
        };
        split2(L.omega, L.omega2);
        split2(L.gfac, L.gfac2);
        for (int k = 0; k < 3; ++k) split2(L.body[k], L.body2[k]);
        const size_t nodes = (size_t)ld->nx * ld->ny * ld->nz;
        h->lbm_nodes = (int64_t)nodes;
        const size_t fb = 19 * nodes * (L.fp32 ? 4 : 8);
        size_t lo = 0;
        auto ltake = [&](size_t bytes) {
            size_t o = lo;
            lo += (bytes + 255) & ~size_t(255);
            return o;
        };
        const size_t o_f0 = ltake(fb), o_f1 = ltake(fb), o_F = ltake(3 * nodes * 8), o_U = ltake(3 * nn * 8),
                     o_c = ltake(nn), o_sc = ltake(4 * nodes * 8);
        if (cudaMalloc(&h->lbm_mem, lo) != cudaSuccess) {
            cudaGetLastError();
            h->err = "device allocation of " + std::to_string(lo) + " bytes for the fluid failed";
            return bail(BPM_ERR_CUDA);
        }
        char* M = (char*)h->lbm_mem;
        L.f[0] = M + o_f0;
        L.f[1] = M + o_f1;
        L.F = M + o_F;
        L.U = (double*)(M + o_U);
        h->lbm_scratch = (double*)(M + o_sc);
        L.coupled = nullptr;
        bool ok2 = true;
        if (ld->coupled) {
            L.coupled = (const uint8_t*)(M + o_c);
            ok2 = cudaMemcpy((void*)L.coupled, ld->coupled, n, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        // initial fields through the scratch (rho [nodes], u [3 nodes])
        double* r0 = nullptr;
        double* u0 = nullptr;
        if (ok2 && ld->rho0) {
            r0 = h->lbm_scratch;
            ok2 = cudaMemcpy(r0, ld->rho0, nodes * 8, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        if (ok2 && ld->u0) {
            u0 = h->lbm_scratch + nodes;
            ok2 = cudaMemcpy(u0, ld->u0, 3 * nodes * 8, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        if (!ok2 || launch_lbm_init(L, r0, u0, nullptr) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            h->err = "fluid setup failed";
            return bail(BPM_ERR_CUDA);
        }
    }
    s.damping = d->damping;
    s.dt = d->dt;
    s.c = d->mu0_over_4pi;
    Field& fd = s.field;
    for (int k = 0; k < 3; ++k) {
        fd.B[k] = d->B[k];
        fd.e1[k] = d->Brot_e1[k];
        fd.e2[k] = d->Brot_e2[k];
        fd.x0[k] = d->gradB_x0[k];
    }
    fd.rot_amp = d->Brot_amp;
    fd.rot_omega = d->Brot_omega;
    fd.has_grad = 0;
    for (int k = 0; k < 9; ++k) {
        fd.G[k] = d->gradB[k];
        if (d->gradB[k] != 0.0) fd.has_grad = 1;
    }
    fd.n_rods = R;
    fd.B_rod = nullptr;
    if (d->B_rod && R > 0) {
        std::vector<double> br(3 * (size_t)R);
        for (int64_t r = 0; r < R; ++r)
            for (int k = 0; k < 3; ++k) br[(size_t)k * R + r] = d->B_rod[3 * r + k];
        if (cudaMemcpy(h->B_rod_d, br.data(), br.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
            h->err = "upload of B_rod failed";
            return bail(BPM_ERR_CUDA);
        }
        fd.B_rod = h->B_rod_d;
    }
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes == 0 || cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up(s.x, x.data(), 3 * n * 8) && up(s.q, q.data(), 4 * n * 8) && up(s.v, v.data(), 3 * n * 8) &&
              up(s.w, w.data(), 3 * n * 8) && up((void*)s.m_body, mb.data(), 3 * n * 8) &&
              up((void*)s.mass, mass.data(), n * 8) && up((void*)s.inertia, inertia.data(), n * 8) &&
              up((void*)s.inv_mass, inv_mass.data(), n * 8) && up((void*)s.inv_inertia, inv_inertia.data(), n * 8) &&
              up((void*)s.bond, bond.data(), 8 * n * 8) && up(h->q_gauge, qg.data(), 4 * n * 8) &&
              up((void*)s.flags, flags.data(), n) && up((void*)s.rod_of, rod_of.data(), n * 4) &&
              up(s.tdev, &d->t0, 8);
    if (!ok || cudaMemset(s.err, 0, 4) != cudaSuccess || cudaMemset(s.step_counter, 0, 4) != cudaSuccess ||
        cudaMemset(h->counter_d, 0, 4) != cudaSuccess || cudaMemset(h->nslot_d, 0, nn) != cudaSuccess ||
        cudaMemset(s.f, 0, 3 * nn * 8) != cudaSuccess || cudaMemset(s.t, 0, 3 * nn * 8) != cudaSuccess) {
        h->err = "initial upload failed";
        return bail(BPM_ERR_CUDA);
    }
    if (cudaMallocHost(&h->pinned_err, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost(&h->pinned_e, sizeof(double) * 8) != cudaSuccess) {
        h->err = "pinned allocation failed";
        return bail(BPM_ERR_CUDA);
    }
    h->cfg.threads = 0;
    h->cfg.blocks = 0;
    if (h->has_lbm && (launch_ibm_interp(s, h->lbm, 0, h->stream) != cudaSuccess ||
                       cudaStreamSynchronize(h->stream) != cudaSuccess)) {
        h->err = "fluid interpolation failed";
        return bail(BPM_ERR_CUDA);
    }
    *out = h;
    return BPM_OK;
}

}  // namespace

extern "C" {

int bpm_create(const bpm_desc* d, bpm_handle** out) { return create_impl(d, nullptr, out); }

int bpm_create_device(const bpm_desc* d, const bpm_device_state* st, bpm_handle** out) {
    if (!st) {
        if (out) *out = nullptr;
        return fail(nullptr, BPM_ERR_ARG, "bpm_create_device: st is NULL");
    }
    return create_impl(d, st, out);
}

void bpm_destroy(bpm_handle* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    if (h->items_d) cudaFree(h->items_d);
    if (h->part_d) cudaFree(h->part_d);
    if (h->adj_arena) cudaFree(h->adj_arena);
    if (h->lbm_mem) cudaFree(h->lbm_mem);
    if (h->arena) cudaFree(h->arena);
    if (h->pinned_err) cudaFreeHost(h->pinned_err);
    if (h->pinned_e) cudaFreeHost(h->pinned_e);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int bpm_forces(bpm_handle* h, double* f, double* tau) {
    if (!h) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    int rc = compute_forces(h, false);
    if (!rc) rc = queue_overflow_read(h);
    if (!rc && f) rc = download_aos(h, h->sys.f, f, 3, nullptr);
    if (!rc && tau) rc = download_aos(h, h->sys.t, tau, 3, nullptr);
    if (!rc) rc = collect_timing(h, false);
    if (!rc) CK(cudaStreamSynchronize(h->stream));
    if (!rc) rc = check_overflow(h);
    return rc;
}

int bpm_step(bpm_handle* h, int32_t nsteps) {
    if (!h) return BPM_ERR_ARG;
    if (nsteps < 0) return fail(h, BPM_ERR_ARG, "bpm_step: n < 0");
    if (nsteps == 0 || h->n == 0) return BPM_OK;
    CK(cudaSetDevice(h->device));
    int rc = BPM_OK;
    if (!h->forces_valid) rc = compute_forces(h, false);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->sys.err, 0, sizeof(int), h->stream));
    CK(cudaMemcpyAsync(h->pinned_err + 1, h->sys.step_counter, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(timed(h, 2, (double)h->n, [&] { return launch_first_half(h->sys, h->stream); }));
    if (h->has_lbm) {
        // LBM cycles: interpolate at the first step of a cycle, one LBM step
        // after every n_sub steps (host-side phase; graphs of single steps)
        if (!h->timing) {
            rc = ensure_graphs(h);
            if (rc) return rc;
        }
        Lbm& L = h->lbm;
        for (int k = 0; k < nsteps && !rc; ++k) {
            const bool last = k + 1 == nsteps;
            if (h->lbm_phase == 0)
                CK(timed(h, 2, (double)h->n, [&] { return launch_ibm_interp(h->sys, L, h->lbm_parity, h->stream); }));
            if (h->timing)
                rc = launch_forces_like(h, last ? FINISH_HALF_KICK : FINISH_CONTINUE, false, true);
            else
                CK(cudaGraphLaunch(last ? h->g_last : h->g_one, h->stream));
            if (rc) return rc;
            if (++h->lbm_phase == L.n_sub) {
                CK(timed(h, 4, (double)h->lbm_nodes, [&] { return launch_lbm_step(L, h->lbm_parity, h->stream); }));
                h->lbm_parity ^= 1;
                h->lbm_phase = 0;
            }
        }
    } else if (h->timing) {
        for (int k = 0; k < nsteps && !rc; ++k)
            rc = launch_forces_like(h, k + 1 == nsteps ? FINISH_HALF_KICK : FINISH_CONTINUE, false, true);
        if (rc) return rc;
    } else {
        rc = ensure_graphs(h);
        if (rc) return rc;
        int rem = nsteps - 1;
        while (rem >= kChunkSteps) {
            CK(cudaGraphLaunch(h->g_chunk, h->stream));
            rem -= kChunkSteps;
        }
        while (rem > 0) {
            CK(cudaGraphLaunch(h->g_one, h->stream));
            --rem;
        }
        CK(cudaGraphLaunch(h->g_last, h->stream));
    }
    CK(cudaMemcpyAsync(h->pinned_err, h->sys.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    rc = queue_overflow_read(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    rc = collect_timing(h, false);
    if (rc) return rc;
    rc = check_overflow(h);
    if (rc) return rc;
    h->forces_valid = true;
    if (h->pinned_err[0] != 0) {
        h->forces_valid = false;
        const int step = h->pinned_err[0] - 1 - h->pinned_err[1];
        return fail(h, BPM_ERR_NONFINITE,
                    "non-finite force, torque, position or orientation at step " + std::to_string(step) +
                        " of this bpm_step call");
    }
    return BPM_OK;
}

int bpm_energy(bpm_handle* h, double out[5]) {
    if (!h || !out) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (h->n == 0) {
        for (int k = 0; k < 5; ++k) out[k] = 0.0;
        return BPM_OK;
    }
    int rc = BPM_OK;
    if (!h->tuned && h->dipole_mode != BPM_DIPOLE_OFF) rc = compute_forces(h, false);
    if (rc) return rc;
    bool timing = h->timing;
    h->timing = false;
    rc = launch_forces_like(h, FINISH_FORCES, true, false);
    h->timing = timing;
    if (rc) return rc;
    h->forces_valid = true;
    CK(launch_energy_reduce(h->sys, h->energy_d, h->stream));
    CK(cudaMemcpyAsync(h->pinned_e, h->energy_d, 5 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    rc = queue_overflow_read(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    rc = check_overflow(h);
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) out[k] = h->pinned_e[k];
    return BPM_OK;
}

int bpm_get_state(bpm_handle* h, double* x, double* q, double* v, double* omega, double* t) {
    if (!h) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    int rc = BPM_OK;
    if (x) rc = download_aos(h, h->sys.x, x, 3, nullptr);
    if (!rc && q && h->n > 0) {
        // q = q' q_rest
        double* tmp = h->sys.e_part;  // 5N scratch, free outside bpm_energy
        CK(cudaMemcpyAsync(tmp, h->sys.q, 4 * (size_t)h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        CK(launch_quat_right_mul(tmp, h->q_gauge, h->n, false, false, h->stream));
        rc = download_aos(h, tmp, q, 4, nullptr);
    }
    if (!rc && v) rc = download_aos(h, h->sys.v, v, 3, nullptr);
    if (!rc && omega) rc = download_aos(h, h->sys.w, omega, 3, nullptr);
    if (!rc && t) {
        CK(cudaMemcpyAsync(h->pinned_e + 5, h->sys.tdev, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *t = h->pinned_e[5];
    }
    if (!rc) CK(cudaStreamSynchronize(h->stream));
    return rc;
}

int bpm_set_state(bpm_handle* h, const double* x, const double* q, const double* v, const double* omega,
                  double t) {
    if (!h) return BPM_ERR_ARG;
    if (!std::isfinite(t)) return fail(h, BPM_ERR_ARG, "bpm_set_state: t must be finite");
    CK(cudaSetDevice(h->device));
    int rc = BPM_OK;
    if (x) rc = upload_aos(h, x, h->sys.x, 3);
    if (!rc && q && h->n > 0) {
        rc = upload_aos(h, q, h->sys.q, 4);
        // q' = q q_rest*, normalised
        if (!rc) CK(launch_quat_right_mul(h->sys.q, h->q_gauge, h->n, true, true, h->stream));
    }
    if (!rc && v) rc = upload_aos(h, v, h->sys.v, 3);
    if (!rc && omega) rc = upload_aos(h, omega, h->sys.w, 3);
    if (rc) return rc;
    CK(launch_zero_clamped(h->sys, h->stream));
    // a new state has no recorded bond measures (NaN bytes) or contact histories
    if (h->sys.hist) CK(cudaMemsetAsync(h->sys.hist, 0xFF, 6 * (size_t)h->n * 8, h->stream));
    if (h->sys.ct_valid) CK(cudaMemsetAsync(h->sys.ct_valid, 0, 8, h->stream));
    if (h->has_lbm) {
        h->lbm_phase = 0;
        CK(launch_ibm_interp(h->sys, h->lbm, h->lbm_parity, h->stream));
    }
    h->pinned_e[6] = t;
    CK(cudaMemcpyAsync(h->sys.tdev, h->pinned_e + 6, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->forces_valid = false;
    return BPM_OK;
}

int bpm_set_forces(bpm_handle* h, const double* f, const double* tau) {
    if (!h) return BPM_ERR_ARG;
    if (!f || !tau) return fail(h, BPM_ERR_ARG, "bpm_set_forces: f and tau are required");
    CK(cudaSetDevice(h->device));
    int rc = BPM_OK;
    // the plan must be fixed before the step graphs are captured
    if (!h->tuned && h->dipole_mode != BPM_DIPOLE_OFF && h->n > 0) rc = compute_forces(h, false);
    if (!rc) rc = upload_aos(h, f, h->sys.f, 3);
    if (!rc) rc = upload_aos(h, tau, h->sys.t, 3);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    h->forces_valid = true;
    return BPM_OK;
}

int bpm_get_forces(bpm_handle* h, double* f, double* tau) {
    if (!h) return BPM_ERR_ARG;
    if (!h->forces_valid) return fail(h, BPM_ERR_ARG, "bpm_get_forces: no forces stored for the current state");
    CK(cudaSetDevice(h->device));
    int rc = BPM_OK;
    if (f) rc = download_aos(h, h->sys.f, f, 3, nullptr);
    if (!rc && tau) rc = download_aos(h, h->sys.t, tau, 3, nullptr);
    if (!rc) CK(cudaStreamSynchronize(h->stream));
    return rc;
}

int bpm_set_field(bpm_handle* h, const double* B, const double* B_rod) {
    if (!h) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (B)
        for (int k = 0; k < 3; ++k) h->sys.field.B[k] = B[k];
    if (B_rod && h->R > 0) {
        std::vector<double> br(3 * (size_t)h->R);
        for (int64_t r = 0; r < h->R; ++r)
            for (int k = 0; k < 3; ++k) br[(size_t)k * h->R + r] = B_rod[3 * r + k];
        CK(cudaMemcpyAsync(h->B_rod_d, br.data(), br.size() * 8, cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->sys.field.B_rod = h->B_rod_d;
    }
    destroy_graphs(h);  // the uniform field is a kernel argument
    h->forces_valid = false;
    h->adj_recorded = false;
    return BPM_OK;
}

int bpm_set_dipoles(bpm_handle* h, const double* m_body) {
    if (!h || !m_body) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    if (h->n == 0) return BPM_OK;
    int rc = upload_aos(h, m_body, (double*)h->sys.m_body, 3);
    if (rc) return rc;
    CK(launch_rotate_vec(h->q_gauge, (double*)h->sys.m_body, h->n, false, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->forces_valid = false;
    h->adj_recorded = false;
    return BPM_OK;
}

int bpm_set_dipole_plan(bpm_handle* h, int32_t kind, int32_t param) {
    if (!h) return BPM_ERR_ARG;
    if (kind == BPM_PLAN_ORDERED) {
        if (h->ff) return fail(h, BPM_ERR_ARG, "ordered plan: a BPM_FF handle has the symmetric kernel only");
        if (param < 1) return fail(h, BPM_ERR_ARG, "ordered plan: param must be >= 1");
        if (h->dipole_mode == BPM_DIPOLE_GLOBAL && param > 255)
            return fail(h, BPM_ERR_ARG, "ordered plan: at most 255 j-chunks");
    } else if (kind == BPM_PLAN_SYMMETRIC) {
        if (param < 0 || param > 8) return fail(h, BPM_ERR_ARG, "symmetric plan: param must be in 0..8");
        int64_t Lmax = h->n;
        if (h->dipole_mode == BPM_DIPOLE_PER_ROD) {
            Lmax = 0;
            for (int64_t r = 0; r < h->R; ++r) Lmax = std::max(Lmax, h->offs[(size_t)r + 1] - h->offs[(size_t)r]);
        }
        const int64_t st = sym_span(h, param);
        if (param == 0 && (double)((Lmax + st - 1) / st) * 56.0 * (double)h->n > 2.0e9)
            return fail(h, BPM_ERR_ARG, "symmetric plan 0: its partial sums would exceed 2 GB");
        if ((Lmax + st - 1) / st > 255) return fail(h, BPM_ERR_ARG, "symmetric plan: more than 255 supertiles");
    } else if (kind != BPM_PLAN_AUTO) {
        return fail(h, BPM_ERR_ARG, "unknown plan kind");
    }
    h->plan_kind = kind;
    h->plan_param = param;
    h->tuned = false;
    h->forces_valid = false;
    destroy_graphs(h);  // captured launches carry the old plan
    return BPM_OK;
}

int bpm_adjoint_begin(bpm_handle* h, int32_t n_steps, int32_t checkpoint_every) {
    if (!h) return BPM_ERR_ARG;
    if (n_steps < 1 || checkpoint_every < 1) return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: need n_steps >= 1, checkpoint_every >= 1");
    if (h->mixed)
        return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: no adjoint for BPM_MIXED handles (BPM_FP64 or BPM_FF)");
    if (h->sys.hist) return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: bond damping is not differentiated");
    if (h->has_contact) return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: contact is not differentiated");
    if (h->has_lbm) return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: the fluid coupling is not differentiated");
    if (h->n == 0) return fail(h, BPM_ERR_ARG, "bpm_adjoint_begin: empty system");
    CK(cudaSetDevice(h->device));
    h->adj_recorded = false;
    // the forces of the starting state are evaluated from that state (its
    // damping uses its own velocities), as the reverse sweep recomputes them
    int rc = compute_forces(h, false);
    if (!rc) rc = adj_alloc(h, n_steps, checkpoint_every);
    if (rc) return rc;
    CK(cudaMemsetAsync(h->sys.err, 0, sizeof(int), h->stream));
    rc = snapshot_handle(h, h->adj_ck);
    if (rc) return rc;
    CK(launch_first_half(h->sys, h->stream));
    for (int k = 1; k < n_steps && !rc; ++k) {
        if (k % checkpoint_every == 0) rc = snapshot_handle(h, h->adj_ck + (size_t)(k / checkpoint_every) * h->adj_snap);
        if (!rc) rc = launch_forces_like(h, FINISH_CONTINUE, false, true);
    }
    if (!rc) rc = launch_forces_like(h, FINISH_HALF_KICK, false, true);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h->pinned_err, h->sys.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    h->forces_valid = true;
    if (h->pinned_err[0] != 0) {
        h->forces_valid = false;
        return fail(h, BPM_ERR_NONFINITE, "bpm_adjoint_begin: the trajectory became non-finite");
    }
    h->adj_steps = n_steps;
    h->adj_every = checkpoint_every;
    h->adj_recorded = true;
    return BPM_OK;
}

int bpm_adjoint_end(bpm_handle* h, const double* dL_dx, double* grad_m_body, double* grad_B) {
    if (!h || !dL_dx) return BPM_ERR_ARG;
    if (!h->adj_recorded) return fail(h, BPM_ERR_ARG, "bpm_adjoint_end: no trajectory recorded by bpm_adjoint_begin");
    CK(cudaSetDevice(h->device));
    const int64_t n = h->n;
    const size_t N = (size_t)n, snap = h->adj_snap;
    AdjBuf& A = h->adj;
    // seed: a(x_K) = dL/dx; everything else zero
    for (double* p : {A.aq}) CK(cudaMemsetAsync(p, 0, 4 * N * 8, h->stream));
    for (double* p : {A.av, A.aw, A.aF, A.aT, A.amb, A.aB}) CK(cudaMemsetAsync(p, 0, 3 * N * 8, h->stream));
    int rc = upload_aos(h, dL_dx, A.ax, 3);
    if (rc) return rc;
    const int steps = h->adj_steps, every = h->adj_every;
    const int nseg = (steps + every - 1) / every;
    for (int seg = nseg - 1; seg >= 0 && !rc; --seg) {
        const int k0 = seg * every, k1 = std::min(k0 + every, steps);
        // recompute P_{k0} .. P_{k1} from the checkpoint (bit-identical to the
        // recorded forward: every kernel is deterministic)
        const double* ck = h->adj_ck + (size_t)seg * snap;
        CK(cudaMemcpyAsync(h->adj_seg, ck, snap * 8, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(h->adj_work, ck, snap * 8, cudaMemcpyDeviceToDevice, h->stream));
        Sys w = snap_view(h, h->adj_work);
        for (int k = k0 + 1; k <= k1 && !rc; ++k) {
            if (k == 1) {
                rc = launch_forces_sys(h, w, FINISH_FORCES, false, false);
                if (!rc) CK(launch_first_half(w, h->stream));
            } else {
                rc = launch_forces_sys(h, w, FINISH_CONTINUE, false, false);
            }
            if (!rc)
                CK(cudaMemcpyAsync(h->adj_seg + (size_t)(k - k0) * snap, h->adj_work, snap * 8,
                                   cudaMemcpyDeviceToDevice, h->stream));
        }
        // reverse sweep over the segment
        for (int k = k1; k > k0 && !rc; --k) {
            Sys prev = snap_view(h, h->adj_seg + (size_t)(k - 1 - k0) * snap);
            Sys cur = snap_view(h, h->adj_seg + (size_t)(k - k0) * snap);
            const double kick = k == 1 ? 0.5 * h->sys.dt : h->sys.dt;
            CK(launch_adj_update(prev, cur, A, kick, h->stream));
            CK(launch_adj_phi(prev, A, h->dipole_mode, h->adj_rod_off, h->stream));
        }
    }
    if (rc) return rc;
    if (grad_B) {
        CK(launch_adj_reduce_B(A.aB, n, h->adj_out, h->stream));
        CK(cudaMemcpyAsync(h->pinned_e, h->adj_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int k = 0; k < 3; ++k) grad_B[k] = h->pinned_e[k];
    }
    if (grad_m_body) {
        // the handle stores m~' = q_rest m~ q_rest*: dL/dm~ = q_rest* (dL/dm~') q_rest
        CK(cudaMemcpyAsync(A.mu, A.amb, 3 * N * 8, cudaMemcpyDeviceToDevice, h->stream));
        CK(launch_rotate_vec(h->q_gauge, A.mu, n, true, h->stream));
        rc = download_aos(h, A.mu, grad_m_body, 3, nullptr);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(h->stream));
    return BPM_OK;
}

int bpm_set_overlap(bpm_handle* h, int32_t mode) {
    if (!h) return BPM_ERR_ARG;
    if (mode < -1 || mode > 1) return fail(h, BPM_ERR_ARG, "overlap mode must be -1, 0 or 1");
    h->overlap_mode = mode;
    h->tuned = false;
    h->forces_valid = false;
    destroy_graphs(h);  // captured launches carry the old form
    return BPM_OK;
}
int bpm_get_overlap(bpm_handle* h, int32_t* on, int32_t* dipole_blocks, int32_t* bond_blocks) {
    if (!h || !on || !dipole_blocks || !bond_blocks) return BPM_ERR_ARG;
    *on = h->tuned && h->overlap ? 1 : 0;
    *dipole_blocks = *on ? h->overlap_blocks : 0;
    *bond_blocks = *on ? h->overlap_bond : 0;
    return BPM_OK;
}
int bpm_get_dipole_plan(bpm_handle* h, int32_t* kind, int32_t* param) {
    if (!h || !kind || !param) return BPM_ERR_ARG;
    if (!h->tuned) {
        *kind = BPM_PLAN_AUTO;
        *param = 0;
    } else {
        *kind = h->cfg.sym ? BPM_PLAN_SYMMETRIC : BPM_PLAN_ORDERED;
        *param = h->cfg.sym ? h->cfg.g : h->tuned_split;
    }
    return BPM_OK;
}

int bpm_lbm_fields(bpm_handle* h, double* rho, double* u) {
    if (!h) return BPM_ERR_ARG;
    if (!h->has_lbm) return fail(h, BPM_ERR_ARG, "bpm_lbm_fields: the system has no fluid");
    CK(cudaSetDevice(h->device));
    const size_t nodes = (size_t)h->lbm_nodes;
    double* r = h->lbm_scratch;
    double* uu = h->lbm_scratch + nodes;
    CK(launch_lbm_macro(h->lbm, h->lbm_parity, r, uu, h->stream));
    if (rho) CK(cudaMemcpyAsync(rho, r, nodes * 8, cudaMemcpyDefault, h->stream));
    if (u) CK(cudaMemcpyAsync(u, uu, 3 * nodes * 8, cudaMemcpyDefault, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return BPM_OK;
}

int bpm_set_timing(bpm_handle* h, int32_t enable) {
    if (!h) return BPM_ERR_ARG;
    h->timing = enable != 0;
    for (int k = 0; k < 5; ++k) h->t_ms[k] = h->launches[k] = h->units[k] = 0.0;
    h->ev_used = 0;
    h->ev_kind.clear();
    h->ev_units.clear();
    return BPM_OK;
}

int bpm_get_timing(bpm_handle* h, double out[15]) {
    if (!h || !out) return BPM_ERR_ARG;
    CK(cudaSetDevice(h->device));
    int rc = collect_timing(h);
    if (rc) return rc;
    for (int k = 0; k < 5; ++k) {
        out[3 * k] = h->launches[k];
        out[3 * k + 1] = h->t_ms[k];
        out[3 * k + 2] = h->units[k];
    }
    return BPM_OK;
}

}  // extern "C"
