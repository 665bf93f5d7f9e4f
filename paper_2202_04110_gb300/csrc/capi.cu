// C-ABI entry points (include/pgm.h): graph build and upload, launch planning, the
// flooding LBP run loop, belief read-out and decode.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgm.h"
#include "audit.h"
#include "pgm_internal.h"

using namespace pgm;

namespace {

thread_local std::string g_last_error;

pgm_status fail(pgm_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

pgm_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return PGM_ECUDA;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

int32_t pgm::set_last_error(int32_t code, const std::string &msg) { return fail(code, msg); }

// One sampled iteration of per-launch timing: its first event, then one event after each
// of its nv variable-pass and nf factor-pass launches.
struct ProfGroup {
    uint32_t first;
    uint16_t nv, nf;
};

struct pgm_graph {
    int device = 0;
    int n_sm = 1;
    bool ordered = false;              // allocations stream-ordered on alloc_stream
    bool has_xor = false;              // a logical group of kind PGM_LOGIC_XOR (no adjoint)
    cudaStream_t alloc_stream = nullptr;
    pgm_info info{};
    DevGraph G{};
    Plan P{};
    void *index_mem = nullptr;    // all index arrays and launch segments
    void *scratch_mem = nullptr;  // ping-pong message buffer, belief buffer, status word
    float *m_tmp = nullptr;
    float *b = nullptr;
    float *lr_d = nullptr, *lr_lam = nullptr;  // Plan::lr: log-ratio arrays (lr_slots each)
    float *lr_prm = nullptr;                    // Plan::lr: table differences [3F] (per run)
    // pgm_run_bp_multi buffers for up to ms_cap samples (allocated on first use)
    void *ms_mem = nullptr;
    int32_t ms_cap = 0;
    float2 *ms_ev = nullptr, *ms_Dv = nullptr;
    float *ms_d = nullptr, *ms_lam = nullptr, *ms_prm = nullptr;
    // pgm_run_bp_until: the messages before a chunk's last iteration [ES] and the residual
    // word (device), its host copy (pinned); allocated on first use
    float *until_prev = nullptr;
    unsigned *until_res = nullptr;       // residual bits; the next word counts iterations done
    unsigned *until_res_host = nullptr;  // 2 words (pinned; stream-ordered graphs: until_words)
    unsigned until_words[2] = {0, 0};
    // device-side early-exit runs (conditional while node), keyed by their arguments
    struct CachedUntil {
        const float *log_pot, *evidence;
        float *msgs;
        uint32_t T_bits, damping_bits, tol_bits;
        int32_t check_every, limit;
        bool members;  // pgm_run_bp_until_members
        cudaGraphExec_t exec;
    };
    std::vector<CachedUntil> untils;
    // pgm_run_bp_until_members (allocated on first use): member edge-state offsets [n+1],
    // frozen words, residual words, iterations and residuals [n each], loop state [3]
    // (iterations done, go on, a member active), the previous messages [n_edge_states]
    char *mu_mem = nullptr;
    // pgm_run_bp_batch (allocated on first use): per-member (T, 1 / T, damping, 0) and
    // iteration counts
    char *bm_mem = nullptr;
    float *bm_prm = nullptr;
    int32_t *bm_iters = nullptr;
    // pgm_run_bp_multi on graphs without the joint log-ratio path: per-sample scratch
    char *mse_mem = nullptr;
    size_t mse_bytes = 0;
    int32_t *mu_off = nullptr, *mu_frozen = nullptr, *mu_iters = nullptr;
    unsigned *mu_res = nullptr;
    float *mu_resid = nullptr, *mu_prev = nullptr;
    int *mu_state = nullptr;
    bool force_es = false;  // edge-state iterations only (the members' early exit)
    // pgm_pmp_sample: perturbed evidence for up to pmp_cap samples (allocated on first use)
    float *pmp_ev = nullptr;
    int32_t pmp_cap = 0;
    int64_t lr_slots = 0;
    // pgm_infer_host buffers (allocated on first use)
    void *host_io_mem = nullptr;
    float *io_pot = nullptr, *io_ev = nullptr, *io_msgs = nullptr, *io_bel = nullptr;
    int32_t *io_dec = nullptr;
    // per-launch event timing
    int32_t profiling = 0;  // sampling period in iterations, 0 = off
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    std::vector<ProfGroup> prof_groups;  // sampled iterations of direct launches
    int64_t prof_var_launches = 0, prof_factor_launches = 0;
    std::vector<double> launch_ms;       // summed event time per launch position
    std::vector<int64_t> launch_n;       // sampled launches per position
    int32_t var_launches = 0, factor_launches = 0;
    std::vector<HostMember> members;
    FactorLaunch adj_launch{};      // pgm_grad: enumeration groups of state sum <= 64, thread per factor
    int32_t adj_nc_max = 0;         // largest list of those groups with a shared table (0: none)
    int32_t adj_block_nc_max = 0;   // the same for the block-form adjoint's groups
    int64_t hd_tot_entries = 0;     // float4 tile totals of the high-degree variables
    int64_t hd_vars = 0;            // high-degree variables (their tile tickets)
    size_t tiles_off = 0;           // their tile list in the index memory
    size_t adj_seg_off = (size_t)-1;
    FactorLaunch adj_block_launch{};  // pgm_grad: the larger groups, block form (k_adj_block)
    size_t adj_block_seg_off = (size_t)-1;
    FactorLaunch adj_logic_launch{};  // pgm_grad: logical groups, thread per factor (k_adj_logic)
    size_t adj_logic_seg_off = (size_t)-1;
    int32_t enum_block = 0;  // PGM_OPT_ENUM_BLOCK
    int32_t pair_form = 0;   // PGM_OPT_PAIR_FORM
    // checked mode (PGM_OPT_CHECKED): the audit's work buffer (allocated on first use),
    // the pools' sizes, the last violation found
    int32_t checked = 0;
    char *audit_mem = nullptr;
    int64_t cfg_size = 0, bs_size = 0, paroff_size = 0;
    int32_t bad_array = -1;
    int64_t bad_pos = -1, bad_value = 0;
    std::vector<std::vector<char>> factor_segs_host;  // host copy of each factor launch's segments
    // CUDA graphs of whole pgm_run_bp calls, keyed by their arguments (LRU)
    struct CachedRun {
        const float *log_pot, *evidence;
        float *msgs;
        uint32_t T_bits, damping_bits;
        int32_t n_iters;
        int32_t prof_period;             // per-launch timing captured in the graph (0 = none)
        cudaGraphExec_t exec;
        uint64_t last_use;
        std::vector<cudaEvent_t> ev;     // events recorded by each replay
        std::vector<ProfGroup> groups;   // the sampled iterations among them
        bool pending = false;            // a replay whose times are not collected yet
    };
    // capture in progress: where take_event puts the graph's events
    std::vector<cudaEvent_t> *capture_events = nullptr;
    std::vector<ProfGroup> *capture_groups = nullptr;
    double graph_var_ms = 0.0, graph_factor_ms = 0.0;  // summed over the sampled passes
    int32_t use_cuda_graph = 1;
    int32_t log_ratio_min_iters = 4;  // PGM_OPT_LOG_RATIO
    int32_t small_run = 1;            // PGM_OPT_SMALL_RUN
    cudaStream_t capture_stream = nullptr;
    std::vector<CachedRun> runs;
    // pgm_grad as CUDA graphs (PGM_OPT_CUDA_GRAPH): persistent work buffers and the
    // recorded calls, keyed by their arguments
    void *grad_mem = nullptr;
    size_t grad_bytes = 0;
    struct CachedGrad {
        const float *log_pot, *evidence, *d_beliefs;
        float *d_log_pot, *d_evidence;
        uint32_t T_bits, damping_bits;
        int32_t n_iters, ckpt_every;
        cudaGraphExec_t exec;
    };
    std::vector<CachedGrad> grads;
    uint64_t use_clock = 0;
};

namespace {

// Bump allocator over one host staging buffer mirrored into one device allocation.
struct Packer {
    std::vector<char> host;
    template <class T>
    size_t add(const T *p, size_t n) {
        size_t off = align_up(host.size(), 256);
        host.resize(off + std::max<size_t>(n * sizeof(T), 1));
        if (n) std::memcpy(host.data() + off, p, n * sizeof(T));
        return off;
    }
};

// Lanes that work on one variable: K / 4 for the K-state group kernels (4 states per
// lane), a warp for kVarWarp, else 1 (per block for kVarBlock).
int var_lanes(int kind) {
    switch (kind) {
        case kVarGroup4: return 1;  // K / 4 lanes per variable, 4 states each
        case kVarGroup8: return 2;
        case kVarGroup16: return 4;
        case kVarWarp: return 32;
        default: return 1;
    }
}

// Lanes that work on one factor: K for the K-lane pairwise kernels, 32 for the warp
// logical kernel, else 1.
int lanes_per_factor(int variant) {
    switch (variant) {
        case kPair4: return 4;
        case kPair8: return 8;
        case kPair16: return 16;
        case kPairQ8: return 2;
        case kPairQ16: return 4;
        case kPairD4: case kPairD8: case kPairD16: return 2;  // a thread per direction
        case kLogicWarp: return 32;
        default: return 1;
    }
}

// Log-ratio iterations apply to a binary pairwise graph: every variable binary (edge e's
// states at 2e), every factor a kPair2 factor, no high-degree variable.
bool lr_eligible(const HostLayout &H) {
    bool lr = H.all_binary && H.logic_groups.empty() && !H.enum_groups.empty() && H.ES == 2 * H.E &&
              H.E % 2 == 0 && H.var_bucket[kVarBlock].empty();
    for (const HostEnumGroup &hg : H.enum_groups) lr = lr && hg.variant == kPair2;
    for (int kind = 0; kind < kNumVarKinds; ++kind)
        if (kind != kVarBinary) lr = lr && H.var_bucket[kind].empty();
    return lr && (H.vin_tab4.empty() ? H.E : 4 * H.V) <= INT32_MAX;
}

// Slots of each log-ratio array: 4 per variable with the 4-slot table, else one per edge.
int64_t lr_slot_count(const HostLayout &H) { return H.vin_tab4.empty() ? H.E : 4 * H.V; }

std::vector<int32_t> lr_slot_map(const HostLayout &H) {
    std::vector<int32_t> pos((size_t)H.E, -1);
    if (!H.vin_tab4.empty()) {
        for (int64_t v = 0; v < H.V; ++v)
            for (int k = 0; k < 4; ++k) {
                const int32_t es = H.vin_tab4[4 * v + k];
                if (es >= 0) pos[es >> 1] = (int32_t)(k * H.V + v);
            }
    } else {
        for (int64_t k = 0; k < H.E; ++k) pos[H.vin_es[k] >> 1] = (int32_t)k;
    }
    return pos;
}

// Block-per-factor enumeration launch (kEnumBlock) with `threads` threads: each segment's
// factors per block (one wave of resident blocks for a large group) and threads per output
// state (enough to fill the factor's team, at most the mean list length, more for long lists;
// one with `one_lane`, which keeps the thread-per-factor kernel's summation order, so
// that groups moved from that kernel give the same bits); block ranges; the dynamic
// shared memory.
static int32_t plan_enum_block(EnumSeg *segs, int n_seg, int threads, int n_sm, bool one_lane, int32_t *smem) {
    int32_t blk = 0;
    *smem = 0;
    for (int i = 0; i < n_seg; ++i) {  // the launch's shared memory first (it sets the occupancy)
        const EnumSeg &sg = segs[i];
        const int teams = sg.es_per_fac <= kEnumWarpStateSum ? threads / 32 : 1;
        *smem = std::max(*smem, ((12 * sg.es_per_fac * teams + 15) & ~15) + sg.table_bytes);
    }
    // one wave: as many blocks as are resident at once, spread over the segments
    const int64_t wave = (int64_t)n_sm * enum_block_resident(threads, *smem);
    for (int i = 0; i < n_seg; ++i) {
        EnumSeg &sg = segs[i];
        const int64_t target = std::max<int64_t>(1, wave);
        sg.fpb = (int32_t)std::max<int64_t>(1, (sg.n_fac + target - 1) / target);
        const int64_t mean = (int64_t)sg.arity * sg.n_cfg / std::max(sg.es_per_fac, 1);
        int lanes = 1;
        // (a property of the group, not of the block size: results do not depend on the
        // shape; a team is a warp up to kEnumWarpStateSum, else a 256-thread block)
        const int team = sg.es_per_fac <= kEnumWarpStateSum ? 32 : kEnumBlockThreads;
        while (!one_lane && lanes < 32 && 2 * lanes <= mean && (int64_t)sg.es_per_fac * 2 * lanes <= team)
            lanes *= 2;
        while (!one_lane && lanes < 32 && mean > 8 * lanes) lanes *= 2;
        sg.lanes = lanes;
        sg.ordered = one_lane ? 1 : 0;
        sg.block_begin = blk;
        blk += (sg.n_fac + sg.fpb - 1) / sg.fpb;
    }
    return blk;
}

pgm_status build_plan(const HostLayout &H, pgm_graph *g, Packer &pk, std::vector<size_t> &seg_off,
                      std::vector<int> &seg_kind) {
    // variable pass: one launch per non-empty bucket of variables
    Plan &P = g->P;
    for (int kind = 0; kind < kNumVarKinds; ++kind) {
        const std::vector<int32_t> &bucket = H.var_bucket[kind];
        if (bucket.empty()) continue;
        VarLaunch L{};
        L.kind = kind;
        L.n = (int32_t)bucket.size();
        L.threads = 256;
        L.n_blocks = (kind == kVarBlock) ? L.n : (int32_t)(((int64_t)L.n * var_lanes(kind) + 255) / 256);
        L.dense_binary = H.all_binary ? 1 : 0;
        L.list = nullptr;
        const size_t list_off = H.var_bucket_identity[kind] ? (size_t)-1 : pk.add(bucket.data(), bucket.size());
        if (kind == kVarBlock) {
            // the split form: a block per tile of 2048 edges (single-sample launches)
            std::vector<int4> tiles;
            int32_t first = 0;
            for (size_t i = 0; i < bucket.size(); ++i) {
                const int32_t v = bucket[i];
                const int32_t deg = H.vin_off[v + 1] - H.vin_off[v], K = H.vs_off[v + 1] - H.vs_off[v];
                const int32_t nt = (deg + kVarTile - 1) / kVarTile;
                for (int32_t t = 0; t < nt; ++t) tiles.push_back(make_int4((int32_t)i, t, first, nt));
                first += nt * K;
            }
            g->hd_tot_entries = first;
            g->hd_vars = (int64_t)bucket.size();
            g->tiles_off = pk.add(tiles.data(), tiles.size());
            L.n_tiles = (int32_t)tiles.size();
        }
        P.var.push_back(L);
        seg_off.push_back(list_off);
        seg_kind.push_back(-1);
    }
    // adjoint factor launches: enumeration groups with a state sum up to kMaxStateSum,
    // thread per factor; larger ones in the team layout of the block form
    {
        std::vector<EnumSeg> segs, bsegs;
        int32_t blk = 0;
        for (const HostEnumGroup &hg : H.enum_groups) {
            EnumSeg s = hg.seg;
            if (s.es_per_fac > kMaxStateSum) {
                bsegs.push_back(s);
                continue;
            }
            s.block_begin = blk;
            blk += (s.n_fac + 127) / 128;
            segs.push_back(s);
        }
        g->adj_nc_max = 0;
        for (const EnumSeg &sg : segs)
            if (sg.shared && sg.n_fac > 0) g->adj_nc_max = std::max(g->adj_nc_max, sg.n_cfg);
        g->adj_launch = FactorLaunch{};
        g->adj_launch.variant = kEnumGeneric;
        g->adj_launch.n_seg = (int32_t)segs.size();
        g->adj_launch.n_blocks = blk;
        g->adj_launch.threads = 128;
        g->adj_seg_off = segs.empty() ? (size_t)-1 : pk.add(segs.data(), segs.size());
        g->adj_block_launch = FactorLaunch{};
        g->adj_block_launch.variant = kEnumBlock;
        if (!bsegs.empty()) {
            int32_t unused = 0;
            g->adj_block_launch.n_blocks =
                plan_enum_block(bsegs.data(), (int)bsegs.size(), kEnumBlockThreads, g->n_sm, false, &unused);
            int32_t sm = 0;  // four state-sum arrays per team
            for (const EnumSeg &sg : bsegs)
                sm = std::max(sm, 16 * sg.es_per_fac * (sg.es_per_fac <= kEnumWarpStateSum ? kEnumBlockThreads / 32 : 1));
            g->adj_block_launch.smem = sm;
            g->adj_block_launch.n_seg = (int32_t)bsegs.size();
            g->adj_block_nc_max = 0;
            for (const EnumSeg &sg : bsegs)
                if (sg.shared && sg.n_fac > 0) g->adj_block_nc_max = std::max(g->adj_block_nc_max, sg.n_cfg);
            g->adj_block_launch.threads = kEnumBlockThreads;
            g->adj_block_seg_off = pk.add(bsegs.data(), bsegs.size());
        }
        // logical groups: thread per factor
        std::vector<LogicSeg> lsegs;
        int32_t lblk = 0;
        g->has_xor = false;
        for (const HostLogicGroup &hg : H.logic_groups) {
            LogicSeg ls = hg.seg;
            g->has_xor |= ls.kind == PGM_LOGIC_XOR && ls.n_fac > 0;
            ls.block_begin = lblk;
            lblk += (ls.n_fac + 127) / 128;
            lsegs.push_back(ls);
        }
        g->adj_logic_launch = FactorLaunch{};
        g->adj_logic_launch.variant = kLogicSmall;
        g->adj_logic_launch.n_seg = (int32_t)lsegs.size();
        g->adj_logic_launch.n_blocks = lblk;
        g->adj_logic_launch.threads = 128;
        g->adj_logic_seg_off = lsegs.empty() ? (size_t)-1 : pk.add(lsegs.data(), lsegs.size());
    }
    // factor pass: one launch per variant, all groups of that variant as segments
    for (int variant = 0; variant < kNumFactorVariants; ++variant) {
        FactorLaunch L{};
        L.variant = variant;
        if (variant == kLogicSmall || variant == kLogicWarp) {
            std::vector<LogicSeg> segs;
            int32_t mf = 0;
            for (const HostLogicGroup &hg : H.logic_groups)
                if (hg.variant == variant) mf = std::max(mf, hg.seg.max_fan);
            int threads = 256, per_block = 256;
            size_t smem = 0;
            if (variant == kLogicWarp) {
                threads = 128;
                per_block = 4;
                smem = (size_t)4 * 3 * mf * sizeof(float);
                if (smem > 200 * 1024) {
                    threads = 32;
                    per_block = 1;
                    smem = (size_t)3 * mf * sizeof(float);
                }
                if (smem > 200 * 1024)
                    return fail(PGM_ENOTSUP, "logical factor fan-in above 17066 is not supported");
            }
            int32_t blk = 0;
            for (const HostLogicGroup &hg : H.logic_groups) {
                if (hg.variant != variant) continue;
                LogicSeg s = hg.seg;
                s.block_begin = blk;
                blk += (s.n_fac + per_block - 1) / per_block;
                segs.push_back(s);
            }
            if (segs.empty()) continue;
            L.n_seg = (int32_t)segs.size();
            L.n_blocks = blk;
            L.threads = threads;
            L.smem = (int32_t)smem;
            L.max_fan = mf;
            L.base_variant = variant;
            P.factor.push_back(L);
            seg_off.push_back(pk.add(segs.data(), segs.size()));
            seg_kind.push_back(variant);
            g->factor_segs_host.emplace_back(reinterpret_cast<const char *>(segs.data()),
                                             reinterpret_cast<const char *>(segs.data() + segs.size()));
        } else {
            std::vector<EnumSeg> segs;
            int threads = (variant == kEnumGeneric || variant == kPairT16) ? 128 : 256;
            const int per_block = threads / lanes_per_factor(variant);
            int32_t blk = 0;
            for (const HostEnumGroup &hg : H.enum_groups) {
                if (hg.variant != variant) continue;
                EnumSeg s = hg.seg;
                s.block_begin = blk;
                blk += (s.n_fac + per_block - 1) / per_block;
                segs.push_back(s);
            }
            if (segs.empty()) continue;
            if (variant == kEnumBlock)
                blk = plan_enum_block(segs.data(), (int)segs.size(), threads, g->n_sm, false, &L.smem);
            L.n_seg = (int32_t)segs.size();
            L.n_blocks = blk;
            L.threads = threads;
            L.max_blocks = g->n_sm * 8;
            L.base_variant = variant;
            P.factor.push_back(L);
            seg_off.push_back(pk.add(segs.data(), segs.size()));
            seg_kind.push_back(variant);
            g->factor_segs_host.emplace_back(reinterpret_cast<const char *>(segs.data()),
                                             reinterpret_cast<const char *>(segs.data() + segs.size()));
        }
    }
    P.lr = lr_eligible(H);
    P.lr_blocks = std::max(1, g->n_sm * 8);
    return PGM_OK;
}

// The next timing event: a new event owned by the graph being captured, or the next one
// of the graph's pool for direct launches.
pgm_status take_event(pgm_graph *g, cudaEvent_t *out) {
    if (g->capture_events) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        g->capture_events->push_back(ev);
        *out = ev;
        return PGM_OK;
    }
    if (g->events.size() <= g->events_used) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        g->events.push_back(ev);
    }
    *out = g->events[g->events_used++];
    return PGM_OK;
}

// Adds the durations of recorded sampled iterations to the graph's per-launch totals
// (waits for each iteration's last event).
pgm_status accumulate_groups(pgm_graph *g, const std::vector<cudaEvent_t> &ev, const std::vector<ProfGroup> &groups) {
    for (const ProfGroup &grp : groups) {
        const int n = grp.nv + grp.nf;
        cudaError_t e = cudaEventSynchronize(ev[grp.first + n]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        if ((int)g->launch_ms.size() < n) {
            g->launch_ms.resize(n, 0.0);
            g->launch_n.resize(n, 0);
        }
        for (int i = 0; i < n; ++i) {
            float dt = 0.f;
            cudaEventElapsedTime(&dt, ev[grp.first + i], ev[grp.first + i + 1]);
            g->launch_ms[i] += dt;
            g->launch_n[i] += 1;
            (i < grp.nv ? g->graph_var_ms : g->graph_factor_ms) += dt;
        }
        g->prof_var_launches += grp.nv;
        g->prof_factor_launches += grp.nf;
    }
    return PGM_OK;
}

// Checked mode: the graph's flat index arrays (device pointers) and their ranges.
std::vector<AuditArray> device_audit_arrays(const pgm_graph *g) {
    const DevGraph &G = g->G;
    const int64_t V = G.V, VS = G.VS, E = G.E, ES = G.ES;
    std::vector<AuditArray> a;
    auto add = [&](const int32_t *p, int64_t n, int64_t lo, int64_t hi, int neg, int id) {
        if (p && n > 0) a.push_back(AuditArray{p, n, lo, hi, neg, id});
    };
    add(G.vs_off, V + 1, 0, VS + 1, false, kAuditVsOff);
    add(G.vin_off, V + 1, 0, E + 1, false, kAuditVinOff);
    add(G.vin_es, E, 0, ES, false, kAuditVinEs);
    add(G.edge_vs, E, 0, VS, 2, kAuditEdgeVs);
    add(G.edge_var, E, 0, V, false, kAuditEdgeVar);
    add(reinterpret_cast<const int32_t *>(G.vin_tab4), 4 * V, 0, ES, true, kAuditTab4);
    add(G.lr_pos, E, 0, g->lr_slots, false, kAuditLrPos);
    add(G.paroff_pool, g->paroff_size, 0, E + 1, false, kAuditParOff);
    for (const VarLaunch &L : g->P.var) add(L.list, L.n, 0, V, false, kAuditVarList);
    return a;
}

// Checked mode (PGM_OPT_CHECKED): before a call's kernels, the device audit of every
// index array and group record; a violation is recorded and ends the call with
// PGM_EINVAL before any LBP kernel reads the bad index.
pgm_status checked_gate(pgm_graph *g, void *stream) {
    if (!g->checked) return PGM_OK;
    DeviceGuard dg(g->device);
    const std::vector<AuditArray> flat = device_audit_arrays(g);
    const size_t need = audit_work_bytes(flat.size());
    if (!g->audit_mem && cudaMalloc(&g->audit_mem, need) != cudaSuccess) {
        g->audit_mem = nullptr;
        return fail(PGM_ENOMEM, "cudaMalloc(index audit)");
    }
    std::vector<std::pair<const void *, int>> enums, logics;
    auto add_launch = [&](const FactorLaunch &L) {
        if (!L.segs || L.n_seg <= 0) return;
        if (L.variant == kLogicSmall || L.variant == kLogicWarp) logics.emplace_back(L.segs, L.n_seg);
        else enums.emplace_back(L.segs, L.n_seg);
    };
    for (const FactorLaunch &L : g->P.factor) add_launch(L);
    if (g->adj_launch.segs) enums.emplace_back(g->adj_launch.segs, g->adj_launch.n_seg);
    if (g->adj_block_launch.segs) enums.emplace_back(g->adj_block_launch.segs, g->adj_block_launch.n_seg);
    if (g->adj_logic_launch.segs) logics.emplace_back(g->adj_logic_launch.segs, g->adj_logic_launch.n_seg);
    const DevGraph &G = g->G;
    const AuditSizes z{G.V, G.VS, G.E, G.ES, g->info.n_potentials, g->cfg_size, g->bs_size, g->paroff_size,
                       G.cfg_pool, G.bs_pool, G.paroff_pool};
    int32_t bad = -1;
    int64_t pos = -1;
    cudaError_t e = audit_device(flat, enums, logics, z, G.flags, g->audit_mem, static_cast<cudaStream_t>(stream),
                                 &bad, &pos);
    if (e != cudaSuccess) return cuda_fail(e, "index audit");
    if (bad < 0) return PGM_OK;
    // the offending entry's value, read back for the report
    int64_t value = -1;
    for (const AuditArray &a : flat)
        if (a.id == bad) {
            int32_t v = 0;
            const AuditArray *hit = &a;
            if (bad == kAuditVarList) {  // several lists share the id: the first one holding pos
                hit = nullptr;
                for (const AuditArray &b : flat)
                    if (b.id == bad && pos < b.n) {
                        hit = &b;
                        break;
                    }
            }
            if (hit && cudaMemcpy(&v, hit->p + pos, sizeof v, cudaMemcpyDeviceToHost) == cudaSuccess) value = v;
            break;
        }
    if (bad == kAuditCfg) {
        uint8_t v = 0;
        if (cudaMemcpy(&v, G.cfg_pool + pos, 1, cudaMemcpyDeviceToHost) == cudaSuccess) value = v;
    } else if (bad == kAuditBs) {
        int32_t v = 0;
        if (cudaMemcpy(&v, G.bs_pool + pos, sizeof v, cudaMemcpyDeviceToHost) == cudaSuccess) value = v;
    }
    g->bad_array = bad;
    g->bad_pos = pos;
    g->bad_value = value;
    return fail(PGM_EINVAL, std::string("checked mode: ") + audit_array_name(bad) + " entry " + std::to_string(pos) +
                                " (value " + std::to_string(value) + ") is out of range; nothing was run");
}

pgm_status check_run_args(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                          float damping, int32_t n_iters, const float *msgs) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    if (!(T >= 0.f) || T == __builtin_inff()) return fail(PGM_EINVAL, "T must be finite and >= 0");
    if (!(damping >= 0.f && damping < 1.f)) return fail(PGM_EINVAL, "damping must be in [0, 1)");
    if (n_iters < 0) return fail(PGM_EINVAL, "n_iters must be >= 0");
    if (!evidence) return fail(PGM_EINVAL, "evidence is NULL");
    if (!msgs && g->info.n_edge_states > 0) return fail(PGM_EINVAL, "msgs is NULL");
    if (!log_pot && g->info.n_potentials > 0) return fail(PGM_EINVAL, "log_pot is NULL");
    return PGM_OK;
}

}  // namespace

// Host-side quiet NaN (the residual before any check).
static const float CUDART_NAN_F_HOST = __builtin_nanf("");

extern "C" {

const char *pgm_last_error(void) { return g_last_error.c_str(); }

// Build a graph. With `ordered`, every allocation, copy and free of the graph is
// stream-ordered on `s` (no device-wide synchronisation; used by the serving loop).
static pgm_status build_from_layout(const HostLayout &H, pgm_graph **out, cudaStream_t s, bool ordered);

static pgm_status build_from_descs(const void *const *descs, int n, pgm_graph **out, cudaStream_t s = nullptr,
                                   bool ordered = false) {
    g_last_error.clear();
    if (!out) return fail(PGM_EINVAL, "out is NULL");
    *out = nullptr;
    HostLayout H;
    std::string err = compile_graph(descs, n, &H);
    if (!err.empty()) return fail(PGM_EINVAL, err);
    return build_from_layout(H, out, s, ordered);
}

// Build a graph from a compiled layout (the device part of pgm_build).
static pgm_status build_from_layout(const HostLayout &H, pgm_graph **out, cudaStream_t s, bool ordered) {
    if (!out) return fail(PGM_EINVAL, "out is NULL");
    *out = nullptr;
    pgm_graph *g = new (std::nothrow) pgm_graph();
    if (!g) return fail(PGM_ENOMEM, "host allocation failed");
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) {
        delete g;
        return cuda_fail(ce, "cudaGetDevice");
    }
    if (cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess || g->n_sm < 1)
        g->n_sm = 1;
    Packer pk;
    size_t o_vs = pk.add(H.vs_off.data(), H.vs_off.size());
    size_t o_vin_off = pk.add(H.vin_off.data(), H.vin_off.size());
    size_t o_vin_es = pk.add(H.vin_es.data(), H.vin_es.size());
    size_t o_edge_vs = pk.add(H.edge_vs.data(), H.edge_vs.size());
    size_t o_cfg = pk.add(H.cfg_pool.data(), H.cfg_pool.size());
    size_t o_po = pk.add(H.paroff_pool.data(), H.paroff_pool.size());
    size_t o_bs = pk.add(H.bs_pool.data(), H.bs_pool.size());
    size_t o_ev = H.edge_var.empty() ? 0 : pk.add(H.edge_var.data(), H.edge_var.size());
    size_t o_tab4 = H.vin_tab4.empty() ? 0 : pk.add(H.vin_tab4.data(), H.vin_tab4.size());
    std::vector<size_t> seg_off;
    std::vector<int> seg_kind;
    pgm_status st = build_plan(H, g, pk, seg_off, seg_kind);
    if (st != PGM_OK) {
        delete g;
        return st;
    }
    // log-ratio layout: slot k V + v of the k-th incoming edge of v (4 slots per
    // variable), else the edge's CSR index
    size_t o_lr_pos = 0;
    if (g->P.lr) {
        const std::vector<int32_t> pos = lr_slot_map(H);
        g->lr_slots = lr_slot_count(H);
        o_lr_pos = pk.add(pos.data(), pos.size());
    }
    g->ordered = ordered;
    g->alloc_stream = s;
    char *dmem = nullptr;
    ce = ordered ? cudaMallocAsync(&dmem, pk.host.size(), s) : cudaMalloc(&dmem, pk.host.size());
    if (ce != cudaSuccess) {
        delete g;
        return fail(PGM_ENOMEM, std::string("cudaMalloc(index arrays): ") + cudaGetErrorString(ce));
    }
    ce = ordered ? cudaMemcpyAsync(dmem, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice, s)
                 : cudaMemcpy(dmem, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        if (ordered) cudaFreeAsync(dmem, s);
        else cudaFree(dmem);
        delete g;
        return cuda_fail(ce, "cudaMemcpy(index arrays)");
    }
    g->index_mem = dmem;
    size_t es_bytes = align_up(std::max<int64_t>(H.ES, 1) * sizeof(float), 256);
    size_t vs_bytes = align_up(std::max<int64_t>(H.VS, 1) * sizeof(float), 256);
    size_t hd_bytes = H.var_bucket[kVarBlock].empty() ? 0 : 4 * vs_bytes;
    const size_t lr_bytes = g->P.lr ? align_up((size_t)g->lr_slots * sizeof(float), 256) : 0;
    const size_t prm_bytes = g->P.lr ? align_up((size_t)3 * (H.E / 2) * sizeof(float), 256) : 0;
    const size_t blo_bytes = keeps_b_lo(H) ? vs_bytes : 0;
    const size_t tot_bytes = align_up((size_t)g->hd_tot_entries * sizeof(float4), 256) +
                             align_up((size_t)g->hd_vars * sizeof(int32_t), 256);
    const size_t scratch_bytes = es_bytes + vs_bytes + 256 + hd_bytes + 2 * lr_bytes + prm_bytes + blo_bytes + tot_bytes;
    char *smem = nullptr;
    ce = ordered ? cudaMallocAsync(&smem, scratch_bytes, s) : cudaMalloc(&smem, scratch_bytes);
    if (ce != cudaSuccess) {
        if (ordered) cudaFreeAsync(dmem, s);
        else cudaFree(dmem);
        delete g;
        return fail(PGM_ENOMEM, std::string("cudaMalloc(scratch): ") + cudaGetErrorString(ce));
    }
    g->scratch_mem = smem;
    g->m_tmp = reinterpret_cast<float *>(smem);
    g->b = reinterpret_cast<float *>(smem + es_bytes);
    uint32_t *flags = reinterpret_cast<uint32_t *>(smem + es_bytes + vs_bytes);
    ce = ordered ? cudaMemsetAsync(flags, 0, 256, s) : cudaMemset(flags, 0, 256);
    if (ce != cudaSuccess) {
        pgm_free(g);
        return cuda_fail(ce, "cudaMemset(flags)");
    }
    DevGraph &G = g->G;
    G.V = (int32_t)H.V;
    G.VS = (int32_t)H.VS;
    G.E = (int32_t)H.E;
    G.ES = (int32_t)H.ES;
    G.vs_off = reinterpret_cast<const int32_t *>(dmem + o_vs);
    G.vin_off = reinterpret_cast<const int32_t *>(dmem + o_vin_off);
    G.vin_es = reinterpret_cast<const int32_t *>(dmem + o_vin_es);
    G.edge_vs = reinterpret_cast<const int32_t *>(dmem + o_edge_vs);
    G.cfg_pool = reinterpret_cast<const uint8_t *>(dmem + o_cfg);
    G.paroff_pool = reinterpret_cast<const int32_t *>(dmem + o_po);
    G.bs_pool = reinterpret_cast<const int32_t *>(dmem + o_bs);
    G.edge_var = H.edge_var.empty() ? nullptr : reinterpret_cast<const int32_t *>(dmem + o_ev);
    G.vin_tab4 = H.vin_tab4.empty() ? nullptr : reinterpret_cast<const int4 *>(dmem + o_tab4);
    G.flags = flags;
    G.hd_b = hd_bytes ? reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256) : nullptr;
    G.lr_pos = g->P.lr ? reinterpret_cast<const int32_t *>(dmem + o_lr_pos) : nullptr;
    G.b_lo = blo_bytes ? reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256 + hd_bytes + 2 * lr_bytes +
                                                    prm_bytes)
                       : nullptr;
    G.hd_tot = tot_bytes ? reinterpret_cast<float4 *>(smem + es_bytes + vs_bytes + 256 + hd_bytes + 2 * lr_bytes +
                                                      prm_bytes + blo_bytes)
                         : nullptr;
    G.hd_cnt = g->hd_vars ? reinterpret_cast<int32_t *>(reinterpret_cast<char *>(G.hd_tot) +
                                                        align_up((size_t)g->hd_tot_entries * sizeof(float4), 256))
                          : nullptr;
    if (G.hd_cnt) {  // the tile tickets start at zero (each launch leaves them so)
        ce = ordered ? cudaMemsetAsync(G.hd_cnt, 0, (size_t)g->hd_vars * sizeof(int32_t), s)
                     : cudaMemset(G.hd_cnt, 0, (size_t)g->hd_vars * sizeof(int32_t));
        if (ce != cudaSuccess) {
            pgm_free(g);
            return cuda_fail(ce, "cudaMemset(tile tickets)");
        }
    }
    if (g->P.lr) {
        g->lr_d = reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256 + hd_bytes);
        g->lr_lam = reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256 + hd_bytes + lr_bytes);
        g->lr_prm = reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256 + hd_bytes + 2 * lr_bytes);
    }
    // attach device pointers of the launch lists / segments
    size_t vi = 0, fi = 0;
    int max_smem = 0;
    for (size_t k = 0; k < seg_off.size(); ++k) {
        if (seg_kind[k] < 0) {
            VarLaunch &L = g->P.var[vi++];
            L.list = (seg_off[k] == (size_t)-1) ? nullptr : reinterpret_cast<const int32_t *>(dmem + seg_off[k]);
            if (L.kind == kVarBlock) L.tiles = reinterpret_cast<const int4 *>(dmem + g->tiles_off);
        } else {
            FactorLaunch &L = g->P.factor[fi++];
            L.segs = dmem + seg_off[k];
            max_smem = std::max(max_smem, L.smem);
        }
    }
    if (g->adj_seg_off != (size_t)-1) g->adj_launch.segs = dmem + g->adj_seg_off;
    if (g->adj_block_seg_off != (size_t)-1) g->adj_block_launch.segs = dmem + g->adj_block_seg_off;
    if (g->adj_logic_seg_off != (size_t)-1) g->adj_logic_launch.segs = dmem + g->adj_logic_seg_off;
    ce = prepare_kernels(max_smem);
    if (ce != cudaSuccess) {
        pgm_free(g);
        return cuda_fail(ce, "cudaFuncSetAttribute");
    }
    // ask now, outside any stream capture, whether the device places the cluster form
    if (g->P.lr && g->G.vin_tab4 != nullptr && g->G.V <= kLrClusterMax * kLrSmallMaxV) lr_cluster_size();
    pgm_info &I = g->info;
    I.n_vars = H.V;
    I.n_var_states = H.VS;
    I.n_factors = H.F;
    I.n_edges = H.E;
    I.n_edge_states = H.ES;
    I.n_potentials = H.P;
    I.max_states = H.max_states;
    I.max_degree = H.max_degree;
    I.device_bytes = (int64_t)(pk.host.size() + scratch_bytes);
    for (const VarLaunch &L : g->P.var) g->var_launches += (L.n > 0);
    for (const FactorLaunch &L : g->P.factor) g->factor_launches += (L.n_blocks > 0);
    I.launches_per_iter = g->var_launches + g->factor_launches;
    I.n_members = (int32_t)H.members.size();
    g->members = H.members;
    g->cfg_size = (int64_t)H.cfg_pool.size();
    g->bs_size = (int64_t)H.bs_pool.size();
    g->paroff_size = (int64_t)H.paroff_pool.size();
    *out = g;
    return PGM_OK;
}

pgm_status pgm_build(const pgm_graph_desc *desc, pgm_graph **out) {
    const void *one = desc;
    return build_from_descs(&one, 1, out);
}

}  // extern "C"

pgm_status pgm::build_graph_on_stream(const pgm_graph_desc *desc, cudaStream_t s, pgm_graph **out) {
    const void *one = desc;
    pgm_status st = build_from_descs(&one, 1, out, s, true);
    if (st == PGM_OK) (*out)->use_cuda_graph = 0;
    return st;
}

int64_t pgm::layout_device_bytes(const HostLayout &H) {
    size_t nb = 0;
    for (int kk = 0; kk < kNumVarKinds; ++kk) nb += H.var_bucket_identity[kk] ? 0 : H.var_bucket[kk].size();
    size_t idx = (H.vs_off.size() + H.vin_off.size() + H.vin_es.size() + H.edge_vs.size() +
                  H.paroff_pool.size() + H.bs_pool.size() + H.edge_var.size() + nb + H.vin_tab4.size()) *
                     sizeof(int32_t) +
                 H.cfg_pool.size();
    size_t es_bytes = align_up(std::max<int64_t>(H.ES, 1) * sizeof(float), 256);
    if (lr_eligible(H))  // the slot map, the two log-ratio arrays and the table differences
        idx += H.E * sizeof(int32_t) + 2 * align_up((size_t)lr_slot_count(H) * sizeof(float), 256) +
               align_up((size_t)3 * (H.E / 2) * sizeof(float), 256);
    const size_t vs_bytes = align_up(std::max<int64_t>(H.VS, 1) * sizeof(float), 256);
    // the high-degree variables' tile list (index memory), tile totals and tickets (scratch)
    int64_t n_tiles = 0, tot = 0;
    for (int32_t v : H.var_bucket[kVarBlock]) {
        const int64_t nt = (H.vin_off[v + 1] - H.vin_off[v] + kVarTile - 1) / kVarTile;
        n_tiles += nt;
        tot += nt * (H.vs_off[v + 1] - H.vs_off[v]);
    }
    idx += (size_t)n_tiles * sizeof(int4);
    return (int64_t)(idx + es_bytes + vs_bytes + 256 + (H.var_bucket[kVarBlock].empty() ? 0 : 4 * vs_bytes) +
                     (keeps_b_lo(H) ? vs_bytes : 0) + align_up((size_t)tot * sizeof(float4), 256) +
                     align_up(H.var_bucket[kVarBlock].size() * sizeof(int32_t), 256));
}

pgm_status pgm::build_layout_on_stream(const HostLayout &H, cudaStream_t s, pgm_graph **out) {
    g_last_error.clear();
    pgm_status st = build_from_layout(H, out, s, true);
    if (st == PGM_OK) (*out)->use_cuda_graph = 0;
    return st;
}

extern "C" {


pgm_status pgm_build_batch(const pgm_graph_desc *const *descs, int32_t n, pgm_graph **out) {
    if (n < 1 || !descs) return fail(PGM_EINVAL, "a batch needs n >= 1 descriptions");
    std::vector<const void *> v(descs, descs + n);
    return build_from_descs(v.data(), n, out);
}

pgm_status pgm_batch_member(const pgm_graph *g, int32_t i, pgm_member *m) {
    if (!g || !m) return fail(PGM_EINVAL, "NULL argument");
    if (i < 0 || i >= (int32_t)g->members.size()) return fail(PGM_EINVAL, "member index out of range");
    const HostMember &h = g->members[i];
    m->var_off = h.var_off;
    m->n_vars = h.n_vars;
    m->vs_off = h.vs_off;
    m->n_var_states = h.n_var_states;
    m->edge_off = h.edge_off;
    m->n_edges = h.n_edges;
    m->es_off = h.es_off;
    m->n_edge_states = h.n_edge_states;
    m->pot_off = h.pot_off;
    m->n_potentials = h.n_potentials;
    return PGM_OK;
}

pgm_status pgm_check_desc(const pgm_graph_desc *desc, pgm_info *info) {
    g_last_error.clear();
    if (!info) return fail(PGM_EINVAL, "info is NULL");
    HostLayout H;
    const void *one = desc;
    std::string err = compile_graph(&one, 1, &H);
    if (!err.empty()) return fail(PGM_EINVAL, err);
    std::memset(info, 0, sizeof *info);
    info->n_vars = H.V;
    info->n_var_states = H.VS;
    info->n_factors = H.F;
    info->n_edges = H.E;
    info->n_edge_states = H.ES;
    info->n_potentials = H.P;
    info->max_states = H.max_states;
    info->max_degree = H.max_degree;
    info->n_members = 1;
    info->device_bytes = pgm::layout_device_bytes(H);
    return PGM_OK;
}

static void drop_cached_runs(pgm_graph *g);

void pgm_free(pgm_graph *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    if (g->ordered) {
        if (g->index_mem) cudaFreeAsync(g->index_mem, g->alloc_stream);
        if (g->scratch_mem) cudaFreeAsync(g->scratch_mem, g->alloc_stream);
        if (g->host_io_mem) cudaFreeAsync(g->host_io_mem, g->alloc_stream);
        if (g->until_prev) cudaFreeAsync(g->until_prev, g->alloc_stream);
        g->index_mem = g->scratch_mem = g->host_io_mem = nullptr;
        g->until_prev = nullptr;
        g->until_res_host = nullptr;  // until_words
    } else {
        cudaDeviceSynchronize();
    }
    if (g->index_mem) cudaFree(g->index_mem);
    if (g->scratch_mem) cudaFree(g->scratch_mem);
    if (g->host_io_mem) cudaFree(g->host_io_mem);
    if (g->ms_mem) cudaFree(g->ms_mem);
    if (g->grad_mem) cudaFree(g->grad_mem);
    if (g->pmp_ev) cudaFree(g->pmp_ev);
    if (g->until_prev) cudaFree(g->until_prev);
    if (g->until_res_host) cudaFreeHost(g->until_res_host);
    if (g->mu_mem) cudaFree(g->mu_mem);
    if (g->bm_mem) cudaFree(g->bm_mem);
    if (g->audit_mem) cudaFree(g->audit_mem);
    if (g->mse_mem) cudaFree(g->mse_mem);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    drop_cached_runs(g);
    if (g->capture_stream) cudaStreamDestroy(g->capture_stream);
    delete g;
}

pgm_status pgm_graph_info(const pgm_graph *g, pgm_info *info) {
    if (!g || !info) return fail(PGM_EINVAL, "NULL argument");
    *info = g->info;
    return PGM_OK;
}

// Enqueue n_iters iterations (and the final copy back into msgs) on stream s.
// On binary pairwise graphs (Plan::lr) runs long enough to repay the two conversions
// iterate on log-ratios: msgs is packed into lr_d, the variable pass writes the
// variable-to-factor values to lr_lam, the factor pass updates lr_d in place, and lr_d
// is unpacked into msgs at the end.
static bool log_ratio_run(const pgm_graph *g, int32_t n_iters) {
    return g->P.lr && !g->force_es && g->log_ratio_min_iters > 0 && n_iters >= g->log_ratio_min_iters;
}

// Whether a log-ratio run of this graph is one launch, and whether that launch is the
// cluster form: the option is on, the graph has the 4-slot layout and fits the form's limits.
// Setting 1 takes one block up to kLrBlockAutoV variables, the cluster above; 2 the
// cluster at any size it takes.
static bool small_run_cluster(const pgm_graph *g) {
    const int V = g->G.V, F = g->G.E / 2;
    if (g->small_run == 2) return true;
    return !(lr_block_fits(V, F) && V <= kLrBlockAutoV) && lr_cluster_fits(V, F);
}
static bool small_run_used(const pgm_graph *g) {
    if (g->small_run == 0 || !g->P.lr || g->G.vin_tab4 == nullptr) return false;
    const int V = g->G.V, F = g->G.E / 2;
    return small_run_cluster(g) ? lr_cluster_fits(V, F) : lr_block_fits(V, F);
}

static pgm_status enqueue_iterations(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                                     float damping, int32_t n_iters, float *msgs, cudaStream_t s,
                                     bool profile) {
    float *cur = msgs, *nxt = g->m_tmp;
    const bool lr = log_ratio_run(g, n_iters);
    // per-variable totals of the 4-slot layout in the belief buffer (VS = 2V floats on a
    // binary graph), which log-ratio iterations do not otherwise use
    float *d = g->lr_d, *lam = g->lr_lam;
    float2 *Dv = reinterpret_cast<float2 *>(g->b);
    // a small graph: the whole run in one launch (per-pass profiling keeps the passes)
    if (lr && small_run_used(g) && !(profile && g->profiling > 0)) {
        cudaError_t e = launch_lr_small_run(g->G, g->P, log_pot, evidence, msgs, lam, T, damping, n_iters,
                                            small_run_cluster(g), s);
        if (e != cudaSuccess) return cuda_fail(e, "small-graph run launch");
        return PGM_OK;
    }
    if (lr) {
        cudaError_t e = launch_lr_pack(g->G, msgs, d, s);
        if (e == cudaSuccess) e = launch_lr_params(g->G, g->P, log_pot, g->lr_prm, s);
        if (e != cudaSuccess) return cuda_fail(e, "log-ratio pack launch");
    }
    // per-launch timing: an event before the iteration and one after each launch
    struct HookCtx {
        pgm_graph *g;
        cudaStream_t s;
        unsigned flags;
        int count;
        pgm_status st;
    };
    auto after_launch = [](void *p) {
        HookCtx *c = static_cast<HookCtx *>(p);
        ++c->count;
        if (c->st != PGM_OK) return;
        cudaEvent_t ev = nullptr;
        c->st = take_event(c->g, &ev);
        if (c->st == PGM_OK) cudaEventRecordWithFlags(ev, c->s, c->flags);
    };
    for (int it = 0; it < n_iters; ++it) {
        const bool prof = profile && g->profiling > 0 && (it % g->profiling) == g->profiling - 1;
        // inside a stream capture the records become event nodes of the graph
        HookCtx ctx{g, s, g->capture_events ? (unsigned)cudaEventRecordExternal : (unsigned)cudaEventRecordDefault, 0,
                    PGM_OK};
        const LaunchHook hook{after_launch, &ctx};
        ProfGroup grp{};
        if (prof) {
            grp.first = (uint32_t)(g->capture_events ? g->capture_events->size() : g->events_used);
            cudaEvent_t e0 = nullptr;
            pgm_status ps = take_event(g, &e0);
            if (ps != PGM_OK) return ps;
            cudaEventRecordWithFlags(e0, s, ctx.flags);
        }
        const LaunchHook *h = prof ? &hook : nullptr;
        cudaError_t e = lr ? launch_lr_var_pass(g->G, g->P, evidence, d, Dv, lam, s, h)
                           : launch_var_pass(g->G, g->P, evidence, cur, g->b, kVarIter, nullptr, s, 1, h);
        if (e != cudaSuccess) return cuda_fail(e, "variable pass launch");
        grp.nv = (uint16_t)ctx.count;
        ctx.count = 0;
        e = lr ? launch_lr_factor_pass(g->G, g->P, log_pot, g->lr_prm, Dv, lam, d, T, damping, s, h)
               : launch_factor_pass(g->G, g->P, log_pot, g->b, evidence, cur, nxt, T, damping, s, 1, h);
        if (e != cudaSuccess) return cuda_fail(e, "factor pass launch");
        grp.nf = (uint16_t)ctx.count;
        if (prof) {
            if (ctx.st != PGM_OK) return ctx.st;
            (g->capture_groups ? *g->capture_groups : g->prof_groups).push_back(grp);
        }
        if (!lr) std::swap(cur, nxt);
    }
    if (lr) {
        cudaError_t e = launch_lr_unpack(g->G, d, msgs, s);
        if (e != cudaSuccess) return cuda_fail(e, "log-ratio unpack launch");
    } else if (cur != msgs) {
        cudaError_t e = cudaMemcpyAsync(msgs, cur, (size_t)g->info.n_edge_states * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(msgs)");
    }
    return PGM_OK;
}

static uint32_t float_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, sizeof u);
    return u;
}

// Adds the per-pass times of a cached run's last replay (if not collected yet) to the
// graph's totals; waits for that replay to finish.
static pgm_status collect_run_times(pgm_graph *g, pgm_graph::CachedRun &r) {
    if (!r.pending) return PGM_OK;
    r.pending = false;
    return accumulate_groups(g, r.ev, r.groups);
}

static void destroy_run(pgm_graph::CachedRun &r) {
    cudaGraphExecDestroy(r.exec);
    for (cudaEvent_t e : r.ev) cudaEventDestroy(e);
    r.ev.clear();
}

// The cached CUDA graph of a pgm_run_bp call with these arguments, captured on the
// graph's private stream on first use.
static pgm_status cached_run(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                             float damping, int32_t n_iters, float *msgs, cudaGraphExec_t *out,
                             pgm_graph::CachedRun **run) {
    const uint32_t tb = float_bits(T), db = float_bits(damping);
    for (auto &r : g->runs)
        if (r.log_pot == log_pot && r.evidence == evidence && r.msgs == msgs && r.T_bits == tb &&
            r.damping_bits == db && r.n_iters == n_iters && r.prof_period == g->profiling) {
            r.last_use = ++g->use_clock;
            *out = r.exec;
            *run = &r;
            return PGM_OK;
        }
    if (!g->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    cudaError_t e = cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    std::vector<cudaEvent_t> events;
    std::vector<ProfGroup> groups;
    g->capture_events = &events;
    g->capture_groups = &groups;
    pgm_status st = enqueue_iterations(g, log_pot, evidence, T, damping, n_iters, msgs, g->capture_stream,
                                       g->profiling > 0);
    g->capture_events = nullptr;
    g->capture_groups = nullptr;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->capture_stream, &graph);
    auto drop_events = [&]() {
        for (cudaEvent_t ev : events) cudaEventDestroy(ev);
    };
    if (st != PGM_OK) {
        if (graph) cudaGraphDestroy(graph);
        drop_events();
        return st;
    }
    if (e != cudaSuccess) drop_events();
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        drop_events();
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    if (g->runs.size() >= 8) {
        size_t lru = 0;
        for (size_t i = 1; i < g->runs.size(); ++i)
            if (g->runs[i].last_use < g->runs[lru].last_use) lru = i;
        collect_run_times(g, g->runs[lru]);
        destroy_run(g->runs[lru]);
        g->runs.erase(g->runs.begin() + lru);
    }
    pgm_graph::CachedRun r{log_pot, evidence, msgs, tb, db, n_iters, g->profiling, exec, ++g->use_clock};
    r.ev = std::move(events);
    r.groups = std::move(groups);
    g->runs.push_back(std::move(r));
    *out = exec;
    *run = &g->runs.back();
    return PGM_OK;
}

static void drop_cached_grads(pgm_graph *g);

static void drop_cached_untils(pgm_graph *g) {
    for (auto &u : g->untils) cudaGraphExecDestroy(u.exec);
    g->untils.clear();
}

static void drop_cached_runs(pgm_graph *g) {
    drop_cached_grads(g);
    drop_cached_untils(g);
    for (auto &r : g->runs) {
        collect_run_times(g, r);
        destroy_run(r);
    }
    g->runs.clear();
}

// pgm_run_bp_multi's buffers for S samples: transposed evidence (V S float2), packed
// messages and flagged-variable lam (4V S each), per-variable totals (V S float2), table
// differences (3F S: room for per-sample tables).
static pgm_status ms_reserve(pgm_graph *g, int32_t S) {
    if (g->ms_cap >= S) return PGM_OK;
    const size_t V = (size_t)g->info.n_vars, F = (size_t)g->info.n_edges / 2;
    const size_t b_ev = align_up(V * S * sizeof(float2), 256), b_d = align_up(4 * V * S * sizeof(float), 256);
    const size_t b_prm = align_up(3 * F * S * sizeof(float), 256);
    if (g->ms_mem) {
        cudaError_t e = cudaDeviceSynchronize();  // the old buffers may still be in use
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        cudaFree(g->ms_mem);
        g->ms_mem = nullptr;
        g->ms_cap = 0;
    }
    char *mem = nullptr;
    if (cudaMalloc(&mem, 2 * b_ev + 2 * b_d + b_prm) != cudaSuccess)
        return fail(PGM_ENOMEM, "cudaMalloc(multi-sample buffers)");
    g->ms_mem = mem;
    g->ms_cap = S;
    g->ms_ev = reinterpret_cast<float2 *>(mem);
    g->ms_Dv = reinterpret_cast<float2 *>(mem + b_ev);
    g->ms_d = reinterpret_cast<float *>(mem + 2 * b_ev);
    g->ms_lam = reinterpret_cast<float *>(mem + 2 * b_ev + b_d);
    g->ms_prm = reinterpret_cast<float *>(mem + 2 * b_ev + 2 * b_d);
    return PGM_OK;
}

// Edge-state iterations of many samples of one graph, the samples as the y dimension of
// every launch: they share the index arrays; each has its own ping-pong partner of its
// messages, beliefs and, where the graph uses them, exact leave-one-out and belief-residual
// scratch. Samples run in chunks whose scratch is at most 1 GiB (and at most 65,535).
static pgm_status run_multi_es(pgm_graph *g, int32_t n_samples, const float *log_pot, int32_t pot_per_sample,
                               const float *evidence, float T, float damping, int32_t n_iters, float *msgs,
                               void *stream) {
    const int64_t VS = g->info.n_var_states, ES = g->info.n_edge_states, P = g->info.n_potentials;
    const int64_t hd = g->G.hd_b ? 4 * VS : 0, blo = g->G.b_lo ? VS : 0;
    const int64_t per = 4 * (ES + VS + hd + blo);
    const int64_t chunk = std::min<int64_t>({(int64_t)n_samples, 65535, std::max<int64_t>(1, ((int64_t)1 << 30) / per)});
    if (chunk <= 1) {
        for (int32_t smp = 0; smp < n_samples; ++smp) {
            pgm_status st = pgm_run_bp(g, log_pot + (pot_per_sample ? (size_t)smp * P : 0),
                                       evidence + (size_t)smp * VS, T, damping, n_iters, msgs + (size_t)smp * ES, stream);
            if (st != PGM_OK) return st;
        }
        return PGM_OK;
    }
    const size_t r_mt = align_up((size_t)(chunk * ES) * 4, 256), r_b = align_up((size_t)(chunk * VS) * 4, 256);
    const size_t r_hd = align_up((size_t)(chunk * hd) * 4, 256), r_lo = align_up((size_t)(chunk * blo) * 4, 256);
    const size_t need = r_mt + r_b + r_hd + r_lo;
    if (g->mse_bytes < need) {
        if (g->mse_mem) cudaFree(g->mse_mem);  // (synchronises the device: no launch still uses it)
        g->mse_mem = nullptr;
        g->mse_bytes = 0;
        if (cudaMalloc(&g->mse_mem, need) != cudaSuccess) return fail(PGM_ENOMEM, "cudaMalloc(multi-sample scratch)");
        g->mse_bytes = need;
    }
    float *mt = reinterpret_cast<float *>(g->mse_mem), *bb = reinterpret_cast<float *>(g->mse_mem + r_mt);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int64_t s0 = 0; s0 < n_samples; s0 += chunk) {
        const int S = (int)std::min<int64_t>(chunk, n_samples - s0);
        DevGraph Gs = g->G;
        Gs.s_es = ES;
        Gs.s_vs = VS;
        Gs.s_pot = pot_per_sample ? P : 0;
        Gs.hd_b = hd ? reinterpret_cast<float *>(g->mse_mem + r_mt + r_b) : nullptr;
        Gs.b_lo = blo ? reinterpret_cast<float *>(g->mse_mem + r_mt + r_b + r_hd) : nullptr;
        const float *lp = log_pot + (pot_per_sample ? (size_t)s0 * P : 0);
        const float *ev = evidence + (size_t)s0 * VS;
        float *m0 = msgs + (size_t)s0 * ES, *cur = m0, *nxt = mt;
        for (int it = 0; it < n_iters; ++it) {
            cudaError_t e = launch_var_pass(Gs, g->P, ev, cur, bb, kVarIter, nullptr, s, S);
            if (e == cudaSuccess) e = launch_factor_pass(Gs, g->P, lp, bb, ev, cur, nxt, T, damping, s, S);
            if (e != cudaSuccess) return cuda_fail(e, "multi-sample pass launch");
            std::swap(cur, nxt);
        }
        if (cur != m0) {
            cudaError_t e = cudaMemcpyAsync(m0, cur, (size_t)S * ES * sizeof(float), cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(multi-sample messages)");
        }
    }
    return PGM_OK;
}

pgm_status pgm_run_bp_multi(pgm_graph *g, int32_t n_samples, const float *log_pot, int32_t pot_per_sample,
                            const float *evidence, float T, float damping, int32_t n_iters, float *msgs,
                            void *stream) {
    if (n_samples < 1) return fail(PGM_EINVAL, "n_samples must be >= 1");
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, n_iters, msgs);
    if (st != PGM_OK) return st;
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    if (n_iters == 0 || g->info.n_edge_states == 0) return PGM_OK;
    const int64_t VS = g->info.n_var_states, ES = g->info.n_edge_states, P = g->info.n_potentials;
    const bool ms = log_ratio_run(g, n_iters) && g->G.vin_tab4 != nullptr &&
                    4 * (int64_t)g->info.n_vars * n_samples <= INT32_MAX;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    if (!ms)  // any other graph: edge-state iterations with the samples side by side
        return run_multi_es(g, n_samples, log_pot, pot_per_sample, evidence, T, damping, n_iters, msgs, stream);
    // Samples run together in chunks whose per-iteration exchange arrays (messages and
    // per-variable totals, plus their table differences and evidence) fit in half the
    // L2, so that the factor pass finds them there; a sample that alone needs more runs
    // on its own, as pgm_run_bp (which keeps one sample's arrays in L2).
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device) != cudaSuccess || l2 <= 0) l2 = 64 << 20;
    const int64_t V = g->info.n_vars, F = g->info.n_edges / 2;
    const int64_t per_sample = 4 * 4 * V + 8 * V + 8 * V + (pot_per_sample ? 12 * F : 0);
    const int32_t chunk = (int32_t)std::min<int64_t>(n_samples, (int64_t)l2 / 2 / std::max<int64_t>(per_sample, 1));
    if (chunk <= 1) {
        for (int32_t smp = 0; smp < n_samples; ++smp) {
            st = pgm_run_bp(g, log_pot + (pot_per_sample ? (size_t)smp * P : 0), evidence + (size_t)smp * VS, T,
                            damping, n_iters, msgs + (size_t)smp * ES, stream);
            if (st != PGM_OK) return st;
        }
        return PGM_OK;
    }
    st = ms_reserve(g, chunk);
    if (st != PGM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int32_t s0 = 0; s0 < n_samples; s0 += chunk) {
        const int S = std::min(chunk, n_samples - s0);
        const int Sp = pot_per_sample ? S : 1;
        const float *lp = log_pot + (pot_per_sample ? (size_t)s0 * P : 0);
        const float *ev = evidence + (size_t)s0 * VS;
        float *m = msgs + (size_t)s0 * ES;
        cudaError_t e = launch_ms_prepare(g->G, g->P, S, Sp, P, lp, ev, m, g->ms_ev, g->ms_d, g->ms_prm, s);
        if (e != cudaSuccess) return cuda_fail(e, "multi-sample prepare launch");
        for (int it = 0; it < n_iters; ++it) {
            e = launch_ms_iteration(g->G, g->P, S, Sp, P, lp, g->ms_prm, g->ms_ev, g->ms_d, g->ms_Dv, g->ms_lam, T,
                                    damping, s);
            if (e != cudaSuccess) return cuda_fail(e, "multi-sample iteration launch");
        }
        e = launch_ms_unpack(g->G, S, g->ms_d, m, s);
        if (e != cudaSuccess) return cuda_fail(e, "multi-sample unpack launch");
    }
    return PGM_OK;
}

// One chunk of an early-exit run: n iterations, the last one's messages in msgs and the
// one before in *prev. An even number of edge-state iterations ends its ping-pong in msgs
// with the previous iteration still in the scratch buffer (no copy); otherwise n - 1
// iterations, a copy of the messages into prev_buf, and one more.
static pgm_status enqueue_chunk(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                                int32_t n, float *msgs, float *prev_buf, const float **prev, cudaStream_t s) {
    if (n % 2 == 0 && !log_ratio_run(g, n)) {
        *prev = g->m_tmp;
        return enqueue_iterations(g, log_pot, evidence, T, damping, n, msgs, s, false);
    }
    *prev = prev_buf;
    pgm_status st = PGM_OK;
    if (n > 1) st = enqueue_iterations(g, log_pot, evidence, T, damping, n - 1, msgs, s, false);
    if (st != PGM_OK) return st;
    cudaError_t e = cudaMemcpyAsync(prev_buf, msgs, (size_t)g->info.n_edge_states * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(messages)");
    return enqueue_iterations(g, log_pot, evidence, T, damping, 1, msgs, s, false);
}

// The graph of the full chunks of an early-exit run: the iteration counter set to 0,
// then a conditional while node whose body runs one chunk (enqueue_chunk, the residual)
// and k_until_control, which
// continues the loop while the residual is above tol (or NaN) and fewer than limit
// iterations are done (so the loop ends after at most limit / check_every trips).
static pgm_status cached_until(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                               int32_t check_every, int32_t limit, float tol, float *msgs, cudaGraphExec_t *out) {
    uint32_t tb, db, lb;
    std::memcpy(&tb, &T, sizeof tb);
    std::memcpy(&db, &damping, sizeof db);
    std::memcpy(&lb, &tol, sizeof lb);
    for (auto &u : g->untils)
        if (!u.members && u.log_pot == log_pot && u.evidence == evidence && u.msgs == msgs && u.T_bits == tb &&
            u.damping_bits == db && u.tol_bits == lb && u.check_every == check_every && u.limit == limit) {
            *out = u.exec;
            return PGM_OK;
        }
    if (!g->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    const int64_t ES = g->info.n_edge_states;
    int *done = reinterpret_cast<int *>(g->until_res + 1);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    auto failed = [&](cudaError_t err, const char *what) {
        cudaGraphDestroy(graph);
        return cuda_fail(err, what);
    };
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return failed(e, "cudaGraphConditionalHandleCreate");
    cudaMemsetParams mp{};
    mp.dst = done;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    cudaGraphNode_t n_init = nullptr, n_loop = nullptr;
    e = cudaGraphAddMemsetNode(&n_init, graph, nullptr, 0, &mp);
    if (e != cudaSuccess) return failed(e, "cudaGraphAddMemsetNode");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&n_loop, graph, &n_init, nullptr, 1, &cp);
    if (e != cudaSuccess) return failed(e, "cudaGraphAddNode(while)");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = g->capture_stream;
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return failed(e, "cudaStreamBeginCaptureToGraph");
    const float *prev = nullptr;
    pgm_status st = enqueue_chunk(g, log_pot, evidence, T, damping, check_every, msgs, g->until_prev, &prev, cs);
    if (st == PGM_OK) {
        e = cudaMemsetAsync(g->until_res, 0, sizeof(unsigned), cs);
        if (e == cudaSuccess) e = launch_residual(ES, msgs, prev, g->until_res, g->n_sm, cs);
        if (e == cudaSuccess) e = launch_until_control(h, g->until_res, done, check_every, limit, tol, cs);
        if (e != cudaSuccess) st = cuda_fail(e, "early-exit body");
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (st != PGM_OK) {
        cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return failed(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(early exit)");
    if (g->untils.size() >= 4) {
        cudaGraphExecDestroy(g->untils.front().exec);
        g->untils.erase(g->untils.begin());
    }
    g->untils.push_back({log_pot, evidence, msgs, tb, db, lb, check_every, limit, false, exec});
    *out = exec;
    return PGM_OK;
}

pgm_status pgm_run_bp_until(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                            int32_t max_iters, float tol, int32_t check_every, float *msgs, int32_t *iters_done,
                            float *residual, void *stream) {
    if (iters_done) *iters_done = 0;
    if (residual) *residual = CUDART_NAN_F_HOST;
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, max_iters, msgs);
    if (st != PGM_OK) return st;
    if (check_every < 1) return fail(PGM_EINVAL, "check_every must be >= 1");
    if (!(tol >= 0.f)) return fail(PGM_EINVAL, "tol must be >= 0");
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    const int64_t ES = g->info.n_edge_states;
    if (max_iters == 0 || ES == 0) {
        if (residual && ES == 0) *residual = 0.f;
        return PGM_OK;
    }
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    if (!g->until_prev && g->ordered) {  // stream-ordered, no pinned word (the serving loop)
        char *mem = nullptr;
        if (cudaMallocAsync(&mem, align_up((size_t)ES * sizeof(float), 256) + 256, g->alloc_stream) != cudaSuccess)
            return fail(PGM_ENOMEM, "cudaMallocAsync(residual buffers)");
        g->until_prev = reinterpret_cast<float *>(mem);
        g->until_res = reinterpret_cast<unsigned *>(mem + align_up((size_t)ES * sizeof(float), 256));
        g->until_res_host = g->until_words;
    }
    if (!g->until_prev) {
        char *mem = nullptr;
        if (cudaMalloc(&mem, align_up((size_t)ES * sizeof(float), 256) + 256) != cudaSuccess)
            return fail(PGM_ENOMEM, "cudaMalloc(residual buffers)");
        g->until_prev = reinterpret_cast<float *>(mem);
        g->until_res = reinterpret_cast<unsigned *>(mem + align_up((size_t)ES * sizeof(float), 256));
        if (cudaMallocHost(&g->until_res_host, 2 * sizeof(unsigned)) != cudaSuccess) {
            cudaFree(g->until_prev);
            g->until_prev = nullptr;
            g->until_res = nullptr;
            g->until_res_host = nullptr;
            return fail(PGM_ENOMEM, "cudaMallocHost(residual word)");
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t done = 0;
    float res = CUDART_NAN_F_HOST;
    // With CUDA graphs on, the full chunks run as one graph whose conditional while node
    // repeats a chunk while its residual is above tol: no host round trip per chunk.
    const int32_t limit = (max_iters / check_every) * check_every;
    if (g->use_cuda_graph && !g->ordered && limit > 0) {
        cudaGraphExec_t exec = nullptr;
        st = cached_until(g, log_pot, evidence, T, damping, check_every, limit, tol, msgs, &exec);
        if (st != PGM_OK) return st;
        cudaError_t e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->until_res_host, g->until_res, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "early-exit graph");
        std::memcpy(&res, g->until_res_host, sizeof res);
        done = (int32_t)g->until_res_host[1];
        if (res <= tol || done >= max_iters) {
            if (iters_done) *iters_done = done;
            if (residual) *residual = res;
            return PGM_OK;
        }
    }
    while (done < max_iters) {
        const int32_t n = std::min(check_every, max_iters - done);
        const float *prev = nullptr;
        st = enqueue_chunk(g, log_pot, evidence, T, damping, n, msgs, g->until_prev, &prev, s);
        if (st != PGM_OK) return st;
        cudaError_t e = cudaMemsetAsync(g->until_res, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = launch_residual(ES, msgs, prev, g->until_res, g->n_sm, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->until_res_host, g->until_res, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "residual");
        std::memcpy(&res, g->until_res_host, sizeof res);
        done += n;
        if (res <= tol) break;
    }
    if (iters_done) *iters_done = done;
    if (residual) *residual = res;
    return PGM_OK;
}

// The graph of the full chunks of a members' early-exit run: a conditional while node
// whose body runs one chunk (enqueue_chunk), the per-member residuals, the loop control (which freezes converged
// members and ends the loop when none is active or limit iterations are done) and the
// copy of newly frozen members' messages to the other ping-pong buffer. The caller
// resets the members' state before each launch.
static pgm_status cached_until_members(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                                       float damping, int32_t check_every, int32_t limit, float tol, float *msgs,
                                       cudaGraphExec_t *out) {
    uint32_t tb, db, lb;
    std::memcpy(&tb, &T, sizeof tb);
    std::memcpy(&db, &damping, sizeof db);
    std::memcpy(&lb, &tol, sizeof lb);
    for (auto &u : g->untils)
        if (u.members && u.log_pot == log_pot && u.evidence == evidence && u.msgs == msgs && u.T_bits == tb &&
            u.damping_bits == db && u.tol_bits == lb && u.check_every == check_every && u.limit == limit) {
            *out = u.exec;
            return PGM_OK;
        }
    if (!g->capture_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    const int64_t ES = g->info.n_edge_states;
    const int nm = (int)g->members.size();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
    auto failed = [&](cudaError_t err, const char *what) {
        cudaGraphDestroy(graph);
        return cuda_fail(err, what);
    };
    cudaGraphConditionalHandle h;
    e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return failed(e, "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_loop = nullptr;
    e = cudaGraphAddNode(&n_loop, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return failed(e, "cudaGraphAddNode(while)");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t cs = g->capture_stream;
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return failed(e, "cudaStreamBeginCaptureToGraph");
    const float *prev = nullptr;
    pgm_status st = enqueue_chunk(g, log_pot, evidence, T, damping, check_every, msgs, g->mu_prev, &prev, cs);
    if (st == PGM_OK) {
        e = launch_residual_members(ES, msgs, prev, g->mu_off, nm, g->mu_frozen, g->mu_res, g->n_sm, cs);
        if (e == cudaSuccess)
            e = launch_until_control_members(h, true, g->mu_res, g->mu_frozen, g->mu_iters, g->mu_resid, nm,
                                             g->mu_state, check_every, limit, tol, cs);
        if (e == cudaSuccess) e = launch_freeze_copy(g->mu_frozen, g->mu_off, nm, msgs, g->m_tmp, g->n_sm, cs);
        if (e != cudaSuccess) st = cuda_fail(e, "members' early-exit body");
    }
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(cs, &captured);
    if (st != PGM_OK) {
        cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return failed(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate(members' early exit)");
    if (g->untils.size() >= 4) {
        cudaGraphExecDestroy(g->untils.front().exec);
        g->untils.erase(g->untils.begin());
    }
    g->untils.push_back({log_pot, evidence, msgs, tb, db, lb, check_every, limit, true, exec});
    *out = exec;
    return PGM_OK;
}

// Device state of the per-member runs of a batch (allocated on first use, kept until
// pgm_free): member edge-state offsets, frozen words (zero outside such runs; every
// factor launch checks them from then on), residual words, iterations, residuals, loop
// state and a previous-messages buffer.
static pgm_status ensure_member_state(pgm_graph *g) {
    const int nm = (int)g->members.size();
    const int64_t ES = g->info.n_edge_states;
    if (!g->mu_mem) {
        const size_t a4 = align_up((size_t)(nm + 1) * sizeof(int32_t), 256);
        const size_t total = 5 * a4 + 256 + align_up((size_t)ES * sizeof(float), 256);
        char *mem = nullptr;
        if (cudaMalloc(&mem, total) != cudaSuccess) return fail(PGM_ENOMEM, "cudaMalloc(members' early-exit state)");
        std::vector<int32_t> off(nm + 1);
        for (int m = 0; m < nm; ++m) off[m] = (int32_t)g->members[m].es_off;
        off[nm] = (int32_t)ES;
        if (cudaMemcpy(mem, off.data(), off.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(mem);
            return fail(PGM_ECUDA, "cudaMemcpy(member offsets)");
        }
        g->mu_mem = mem;
        g->mu_off = reinterpret_cast<int32_t *>(mem);
        g->mu_frozen = reinterpret_cast<int32_t *>(mem + a4);
        g->mu_res = reinterpret_cast<unsigned *>(mem + 2 * a4);
        g->mu_iters = reinterpret_cast<int32_t *>(mem + 3 * a4);
        g->mu_resid = reinterpret_cast<float *>(mem + 4 * a4);
        g->mu_state = reinterpret_cast<int *>(mem + 5 * a4);
        g->mu_prev = reinterpret_cast<float *>(mem + 5 * a4 + 256);
        if (cudaMemset(g->mu_frozen, 0, (size_t)nm * sizeof(int32_t)) != cudaSuccess)
            return fail(PGM_ECUDA, "cudaMemset(frozen)");
        g->G.frozen = g->mu_frozen;  // launches from now on check it (zero outside these runs)
    }
    return PGM_OK;
}

pgm_status pgm_run_bp_until_members(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                                    float damping, int32_t max_iters, float tol, int32_t check_every, float *msgs,
                                    int32_t *iters_done, float *residual, void *stream) {
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, max_iters, msgs);
    if (st != PGM_OK) return st;
    if (!iters_done || !residual) return fail(PGM_EINVAL, "iters_done / residual is NULL");
    if (check_every < 1) return fail(PGM_EINVAL, "check_every must be >= 1");
    if (!(tol >= 0.f)) return fail(PGM_EINVAL, "tol must be >= 0");
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    const int nm = (int)g->members.size();
    const int64_t ES = g->info.n_edge_states;
    for (int m = 0; m < nm; ++m) {
        iters_done[m] = 0;
        residual[m] = (max_iters == 0 && g->members[m].n_edge_states > 0) ? CUDART_NAN_F_HOST : 0.f;
    }
    if (max_iters == 0 || ES == 0) return PGM_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    st = ensure_member_state(g);
    if (st != PGM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    struct ForceEs {  // edge-state iterations for the whole call
        pgm_graph *g;
        ~ForceEs() { g->force_es = false; }
    } force{g};
    g->force_es = true;
    cudaError_t e = launch_until_members_init(g->mu_frozen, g->mu_res, g->mu_iters, g->mu_resid, g->mu_off, nm,
                                              g->mu_state, s);
    if (e != cudaSuccess) return cuda_fail(e, "members' early-exit reset");
    int state[3] = {0, 1, 1};  // iterations done, go on, a member active
    const int32_t limit = (max_iters / check_every) * check_every;
    if (g->use_cuda_graph && !g->ordered && limit > 0) {
        cudaGraphExec_t exec = nullptr;
        st = cached_until_members(g, log_pot, evidence, T, damping, check_every, limit, tol, msgs, &exec);
        if (st != PGM_OK) return st;
        e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(state, g->mu_state, sizeof state, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "members' early-exit graph");
    }
    // the rest (all of it with CUDA graphs off): chunks checked by the host
    while (state[0] < max_iters && state[2]) {
        const int32_t n = std::min(check_every, max_iters - state[0]);
        const float *prev = nullptr;
        st = enqueue_chunk(g, log_pot, evidence, T, damping, n, msgs, g->mu_prev, &prev, s);
        if (st != PGM_OK) return st;
        e = launch_residual_members(ES, msgs, prev, g->mu_off, nm, g->mu_frozen, g->mu_res, g->n_sm, s);
        if (e == cudaSuccess)
            e = launch_until_control_members(0, false, g->mu_res, g->mu_frozen, g->mu_iters, g->mu_resid, nm,
                                             g->mu_state, n, max_iters, tol, s);
        if (e == cudaSuccess) e = launch_freeze_copy(g->mu_frozen, g->mu_off, nm, msgs, g->m_tmp, g->n_sm, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(state, g->mu_state, sizeof state, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "members' early exit");
    }
    e = cudaMemcpyAsync(iters_done, g->mu_iters, (size_t)nm * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(residual, g->mu_resid, (size_t)nm * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mu_frozen, 0, (size_t)nm * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "members' early-exit results");
    return PGM_OK;
}

pgm_status pgm_run_bp_batch(pgm_graph *g, const float *log_pot, const float *evidence, const float *T,
                            const float *damping, const int32_t *n_iters, float *msgs, void *stream) {
    pgm_status st = check_run_args(g, log_pot, evidence, 1.f, 0.f, 0, msgs);
    if (st != PGM_OK) return st;
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    if (!T || !damping || !n_iters) return fail(PGM_EINVAL, "T / damping / n_iters is NULL");
    const int nm = (int)g->members.size();
    const int64_t ES = g->info.n_edge_states;
    std::vector<float> prm(4 * (size_t)nm, 0.f);
    int32_t max_it = 0;
    bool any_max = false, any_sum = false, finish_at_zero = false;
    for (int m = 0; m < nm; ++m) {
        if (!(T[m] >= 0.f) || T[m] == __builtin_inff())
            return fail(PGM_EINVAL, "T[" + std::to_string(m) + "] must be finite and >= 0");
        if (!(damping[m] >= 0.f && damping[m] < 1.f))
            return fail(PGM_EINVAL, "damping[" + std::to_string(m) + "] must be in [0, 1)");
        if (n_iters[m] < 0) return fail(PGM_EINVAL, "n_iters[" + std::to_string(m) + "] must be >= 0");
        prm[4 * m] = T[m];
        prm[4 * m + 1] = T[m] > 0.f ? 1.f / T[m] : 0.f;
        prm[4 * m + 2] = damping[m];
        if (g->members[m].n_edge_states == 0) continue;
        if (n_iters[m] == 0) {
            finish_at_zero = true;
            continue;
        }
        max_it = std::max(max_it, n_iters[m]);
        (T[m] == 0.f ? any_max : any_sum) = true;
    }
    if (max_it == 0 || ES == 0) return PGM_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    st = ensure_member_state(g);
    if (st != PGM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!g->bm_mem) {
        const size_t a = align_up((size_t)nm * 4 * sizeof(float), 256);
        if (cudaMalloc(&g->bm_mem, a + align_up((size_t)nm * sizeof(int32_t), 256)) != cudaSuccess) {
            g->bm_mem = nullptr;
            return fail(PGM_ENOMEM, "cudaMalloc(per-member parameters)");
        }
        g->bm_prm = reinterpret_cast<float *>(g->bm_mem);
        g->bm_iters = reinterpret_cast<int32_t *>(g->bm_mem + a);
    }
    // pageable sources: each copy has taken its data when the call returns
    std::vector<int32_t> frozen(nm), iters(n_iters, n_iters + nm);
    for (int m = 0; m < nm; ++m) frozen[m] = (n_iters[m] == 0 || g->members[m].n_edge_states == 0) ? 1 : 0;
    cudaError_t e = cudaMemcpyAsync(g->bm_prm, prm.data(), prm.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->bm_iters, iters.data(), iters.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->mu_frozen, frozen.data(), frozen.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "per-member parameters upload");
    DevGraph G2 = g->G;
    G2.mem_prm = g->bm_prm;
    G2.frozen = g->mu_frozen;
    float *cur = msgs, *nxt = g->m_tmp;
    // members that run no iteration: both buffers hold their messages
    if (finish_at_zero) e = launch_batch_freeze(g->bm_iters, 0, nm, g->mu_off, g->mu_frozen, cur, nxt, g->n_sm, s);
    std::vector<char> ends((size_t)max_it + 1, 0);
    for (int m = 0; m < nm; ++m)
        if (n_iters[m] > 0 && g->members[m].n_edge_states > 0) ends[n_iters[m]] = 1;
    for (int32_t it = 0; it < max_it && e == cudaSuccess; ++it) {
        e = launch_var_pass(G2, g->P, evidence, cur, g->b, kVarIter, nullptr, s);
        // one launch per kind of member: max-product (T = 0) and the others
        if (e == cudaSuccess && any_max) e = launch_factor_pass(G2, g->P, log_pot, g->b, evidence, cur, nxt, 0.f, 0.f, s);
        if (e == cudaSuccess && any_sum) e = launch_factor_pass(G2, g->P, log_pot, g->b, evidence, cur, nxt, 1.f, 0.f, s);
        std::swap(cur, nxt);
        if (e == cudaSuccess && ends[it + 1] && it + 1 < max_it)
            e = launch_batch_freeze(g->bm_iters, it + 1, nm, g->mu_off, g->mu_frozen, cur, nxt, g->n_sm, s);
    }
    if (e == cudaSuccess && cur != msgs)
        e = cudaMemcpyAsync(msgs, cur, (size_t)ES * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mu_frozen, 0, (size_t)nm * sizeof(int32_t), s);
    // the host vectors above are the copies' sources: keep them until the copies are done
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "batch run with per-member parameters");
    return PGM_OK;
}

pgm_status pgm_pmp_sample(pgm_graph *g, int32_t n_samples, const float *log_pot, const float *evidence,
                          const float *noise, float damping, int32_t n_iters, float *msgs, int32_t *samples,
                          void *stream) {
    if (n_samples < 1) return fail(PGM_EINVAL, "n_samples must be >= 1");
    if (!noise || !samples) return fail(PGM_EINVAL, "noise / samples is NULL");
    pgm_status st = check_run_args(g, log_pot, evidence, 0.f, damping, n_iters, msgs);
    if (st != PGM_OK) return st;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    const int64_t VS = g->info.n_var_states, ES = g->info.n_edge_states, V = g->info.n_vars;
    if (g->pmp_cap < n_samples) {
        if (g->pmp_ev) {
            cudaError_t e = cudaDeviceSynchronize();  // the old buffer may still be in use
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            cudaFree(g->pmp_ev);
            g->pmp_ev = nullptr;
            g->pmp_cap = 0;
        }
        if (cudaMalloc(&g->pmp_ev, (size_t)VS * n_samples * sizeof(float)) != cudaSuccess) {
            g->pmp_ev = nullptr;
            return fail(PGM_ENOMEM, "cudaMalloc(perturbed evidence)");
        }
        g->pmp_cap = n_samples;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pmp_perturb(VS, n_samples, evidence, noise, g->pmp_ev, s);
    if (e == cudaSuccess && ES > 0) e = cudaMemsetAsync(msgs, 0, (size_t)ES * n_samples * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "perturb-and-max-product set-up");
    st = pgm_run_bp_multi(g, n_samples, log_pot, 0, g->pmp_ev, 0.f, damping, n_iters, msgs, stream);
    if (st != PGM_OK) return st;
    for (int32_t smp = 0; smp < n_samples; ++smp) {
        e = launch_var_pass(g->G, g->P, g->pmp_ev + (size_t)smp * VS, msgs + (size_t)smp * ES, nullptr, kVarDecode,
                            samples + (size_t)smp * V, s);
        if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    }
    return PGM_OK;
}

pgm_status pgm_run_bp(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                      float damping, int32_t n_iters, float *msgs, void *stream) {
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, n_iters, msgs);
    if (st != PGM_OK) return st;
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    if (n_iters == 0 || g->info.n_edge_states == 0) return PGM_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g->use_cuda_graph && n_iters >= 2) {
        cudaGraphExec_t exec = nullptr;
        pgm_graph::CachedRun *run = nullptr;
        st = cached_run(g, log_pot, evidence, T, damping, n_iters, msgs, &exec, &run);
        if (st != PGM_OK) return st;
        st = collect_run_times(g, *run);  // the previous replay's times, before they are overwritten
        if (st != PGM_OK) return st;
        cudaError_t e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        run->pending = !run->groups.empty();
        return PGM_OK;
    }
    return enqueue_iterations(g, log_pot, evidence, T, damping, n_iters, msgs, s, true);
}

// The other kernel forms for the same factors: dense K-state pairwise tables run with K
// lanes per factor (kPair4 / 8 / 16), a thread per factor (kPairT4 / 8 / 16) or, for
// tables shared by the group, K / 4 lanes per factor (kPairQ8 / 16).
static std::vector<int> alternative_forms(int base_variant, bool all_shared) {
    switch (base_variant) {
        case kPair4: case kPairT4: case kPairD4: return {kPairT4, kPairD4, kPair4};
        case kPair8: case kPairT8: case kPairQ8: case kPairD8:
            return all_shared ? std::vector<int>{kPairT8, kPairD8, kPairQ8, kPair8}
                              : std::vector<int>{kPairT8, kPairD8, kPair8};
        case kPair16: case kPairT16: case kPairQ16: case kPairD16:
            return all_shared ? std::vector<int>{kPairT16, kPairD16, kPairQ16, kPair16}
                              : std::vector<int>{kPairT16, kPairD16, kPair16};
        case kEnumGeneric: case kEnumBlock: return {kEnumGeneric, kEnumBlock};  // the former where every group fits
        default: return {base_variant};
    }
}

// Thread-block shapes a factor launch may use (within the kernels' launch bounds).
static std::vector<int> shape_candidates(int variant) {
    switch (variant) {
        case kPair2: case kPair4: case kPair8: case kPair16: case kLogicSmall: return {64, 128, 256};
        case kPairT4: case kPairT8: return {64, 128, 256};
        case kPairT16: return {64, 128};
        case kPairQ8: case kPairQ16: return {64, 128, 256};
        case kPairD4: case kPairD8: case kPairD16: return {64, 128, 256};  // warp pairs
        case kEnumGeneric: return {32, 64, 128};
        case kEnumBlock: return {128, 256};
        case kLogicWarp: return {32, 64, 128};
        default: return {};
    }
}

// Re-plan factor launch li for `threads` threads per block: block ranges of its segments,
// grid size, shared memory; uploads the segments. Returns false if the shape does not fit.
static bool replan_factor_launch(pgm_graph *g, size_t li, int threads, cudaStream_t s) {
    FactorLaunch &L = g->P.factor[li];
    std::vector<char> &host = g->factor_segs_host[li];
    const bool logic = (L.variant == kLogicSmall || L.variant == kLogicWarp);
    const int per_block = threads / lanes_per_factor(L.variant);
    size_t smem = 0;
    if (L.variant == kLogicWarp) {
        smem = (size_t)per_block * 3 * L.max_fan * sizeof(float);
        if (smem > 200 * 1024) return false;
    }
    int32_t blk = 0;
    if (logic) {
        LogicSeg *segs = reinterpret_cast<LogicSeg *>(host.data());
        for (int i = 0; i < L.n_seg; ++i) {
            segs[i].block_begin = blk;
            blk += (segs[i].n_fac + per_block - 1) / per_block;
        }
    } else if (L.variant == kEnumBlock) {
        int32_t sm = 0;
        blk = plan_enum_block(reinterpret_cast<EnumSeg *>(host.data()), L.n_seg, threads, g->n_sm,
                              L.base_variant == kEnumGeneric, &sm);
        smem = (size_t)sm;
        if (prepare_kernels(sm) != cudaSuccess) return false;
    } else {
        EnumSeg *segs = reinterpret_cast<EnumSeg *>(host.data());
        for (int i = 0; i < L.n_seg; ++i) {
            if (L.variant == kEnumGeneric && segs[i].es_per_fac > kMaxStateSum) return false;
            segs[i].block_begin = blk;
            blk += (segs[i].n_fac + per_block - 1) / per_block;
        }
    }
    if (cudaMemcpyAsync(const_cast<void *>(L.segs), host.data(), host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return false;
    L.threads = threads;
    L.n_blocks = blk;
    L.smem = (int32_t)smem;
    return true;
}

pgm_status pgm_autotune(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                        float damping, void *stream) {
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, 1, g ? g->m_tmp : nullptr);
    if (st != PGM_OK) return st;
    if ((st = checked_gate(g, stream)) != PGM_OK) return st;
    if (g->info.n_edge_states == 0) return PGM_OK;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t es_bytes = (size_t)g->info.n_edge_states * sizeof(float);
    float *m_in = nullptr, *m_out = nullptr;
    if (cudaMalloc(&m_in, 2 * es_bytes) != cudaSuccess) return fail(PGM_ENOMEM, "cudaMalloc(autotune buffers)");
    m_out = m_in + g->info.n_edge_states;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaMemsetAsync(m_in, 0, es_bytes, s);
    // one real iteration so that the messages and beliefs are not trivial
    enqueue_iterations(g, log_pot, evidence, T, damping, 1, m_in, s, false);
    launch_var_pass(g->G, g->P, evidence, m_in, g->b, kVarIter, nullptr, s);
    for (size_t li = 0; li < g->P.factor.size(); ++li) {
        const int orig_variant = g->P.factor[li].variant;
        int best = g->P.factor[li].threads, best_variant = orig_variant;
        float best_ms = 1e30f;
        // the kernel forms that can run this launch's groups, each with its block shapes
        bool all_shared = true;
        {
            const FactorLaunch &L0 = g->P.factor[li];
            if (L0.variant != kLogicSmall && L0.variant != kLogicWarp) {
                const EnumSeg *segs = reinterpret_cast<const EnumSeg *>(g->factor_segs_host[li].data());
                for (int i = 0; i < L0.n_seg; ++i) all_shared = all_shared && segs[i].shared != 0;
            }
        }
        const std::vector<int> forms = alternative_forms(g->P.factor[li].base_variant, all_shared);
        for (int variant : forms) {
            g->P.factor[li].variant = variant;
            for (int c : shape_candidates(variant)) {
                if (!replan_factor_launch(g, li, c, s)) continue;
                Plan one;
                one.factor.push_back(g->P.factor[li]);
                launch_factor_pass(g->G, one, log_pot, g->b, evidence, m_in, m_out, T, damping, s);
                cudaEventRecord(e0, s);
                for (int r = 0; r < 5; ++r)
                    launch_factor_pass(g->G, one, log_pot, g->b, evidence, m_in, m_out, T, damping, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (cudaGetLastError() == cudaSuccess && ms < best_ms) {
                    best_ms = ms;
                    best = c;
                    best_variant = variant;
                }
            }
        }
        g->P.factor[li].variant = best_variant;
        replan_factor_launch(g, li, best, s);
    }
    // thread-per-variable launches: block size
    for (VarLaunch &L : g->P.var) {
        if (L.kind == kVarBlock || L.n == 0 || g->G.vin_tab4) continue;
        int best = L.threads;
        float best_ms = 1e30f;
        for (int c : {128, 256}) {
            L.threads = c;
            L.n_blocks = (int32_t)(((int64_t)L.n * var_lanes(L.kind) + c - 1) / c);
            Plan one;
            one.var.push_back(L);
            launch_var_pass(g->G, one, evidence, m_in, g->b, kVarIter, nullptr, s);
            cudaEventRecord(e0, s);
            for (int r = 0; r < 5; ++r) launch_var_pass(g->G, one, evidence, m_in, g->b, kVarIter, nullptr, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        L.threads = best;
        L.n_blocks = (int32_t)(((int64_t)L.n * var_lanes(L.kind) + best - 1) / best);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(m_in);
    drop_cached_runs(g);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    return PGM_OK;
}

pgm_status pgm_launch_info(const pgm_graph *g, int32_t i, int32_t *kind, int32_t *variant,
                           int32_t *threads, int32_t *n_blocks) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    const int32_t nv = (int32_t)g->P.var.size(), nf = (int32_t)g->P.factor.size();
    if (i < 0 || i >= nv + nf) return fail(PGM_EINVAL, "launch index out of range");
    if (i < nv) {
        const VarLaunch &L = g->P.var[i];
        if (kind) *kind = 0;
        if (variant) *variant = g->G.vin_tab4 ? 6 : (L.kind == kVarWarp ? 7 : L.kind);
        if (threads) *threads = L.kind == kVarBlock ? kVarBlockThreads : (g->G.vin_tab4 ? 256 : L.threads);
        if (n_blocks)
            *n_blocks = g->G.vin_tab4 ? (int32_t)((g->info.n_vars + 255) / 256)
                                      : (L.kind == kVarBlock ? L.n_tiles : L.n_blocks);
    } else {
        const FactorLaunch &L = g->P.factor[i - nv];
        if (kind) *kind = 1;
        if (variant) *variant = L.variant;
        if (threads) *threads = L.threads;
        if (n_blocks) *n_blocks = L.n_blocks;
    }
    return PGM_OK;
}

// One iteration from `in` into `out` (out != in).
static pgm_status one_iteration(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                                const float *in, float *out, cudaStream_t s) {
    cudaError_t e = launch_var_pass(g->G, g->P, evidence, in, g->b, kVarIter, nullptr, s);
    if (e == cudaSuccess) e = launch_factor_pass(g->G, g->P, log_pot, g->b, evidence, in, out, T, damping, s);
    if (e != cudaSuccess) return cuda_fail(e, "iteration launch");
    return PGM_OK;
}

// The warp partials of shared-table gradients (k_adj_factor): warps of the launch x the
// largest shared list.
static size_t grad_partials_bytes(const pgm_graph *g) {
    if (g->adj_nc_max == 0) return 0;
    return align_up((size_t)g->adj_launch.n_blocks * (g->adj_launch.threads / 32) * g->adj_nc_max * sizeof(float), 256);
}

// The variable pass's outputs of one recomputed iteration, kept for its reverse step: the
// beliefs, and the high-degree totals and belief residuals where the graph has them.
static size_t grad_step_bytes(const pgm_graph *g) {
    const size_t vsb = align_up((size_t)std::max<int64_t>(g->info.n_var_states, 1) * sizeof(float), 256);
    return vsb * (1 + (g->G.hd_b ? 4 : 0) + (g->G.b_lo ? 1 : 0));
}

// The team rows of block-form shared-table gradients (k_adj_block): blocks x 8 teams x the
// largest such list; 0 (the kernel then adds with atomics) beyond 512 MiB.
static size_t grad_block_partials_bytes(const pgm_graph *g) {
    if (g->adj_block_nc_max == 0 || g->adj_block_launch.n_blocks == 0) return 0;
    const size_t b = align_up((size_t)g->adj_block_launch.n_blocks * (kEnumBlockThreads / 32) *
                                  (size_t)g->adj_block_nc_max * sizeof(float), 256);
    return b <= ((size_t)512 << 20) ? b : 0;
}

// Whether a gradient keeps each recomputed iteration's variable-pass outputs (so that its
// reverse step launches no variable pass): when one segment's worth fits in 256 MiB.
static bool grad_keeps_steps(const pgm_graph *g, int32_t n_iters, int32_t ckpt_every) {
    const int seg_len = std::min(ckpt_every, std::max(n_iters, 1));
    return (size_t)seg_len * grad_step_bytes(g) <= ((size_t)256 << 20);
}

// Work buffers of a gradient: checkpoints, one segment of recomputed states, two message
// buffers, two adjoint buffers, the variable-to-factor adjoint, the damping adjoint, the
// warp partials of shared-table gradients, and the kept variable-pass outputs.
static size_t grad_work_bytes(const pgm_graph *g, int32_t n_iters, int32_t ckpt_every) {
    const int64_t ES = std::max<int64_t>(g->info.n_edge_states, 1);
    const size_t esb = align_up((size_t)ES * sizeof(float), 256);
    const int n_ck = n_iters > 0 ? (n_iters + ckpt_every - 1) / ckpt_every : 0;
    const int seg_len = std::min(ckpt_every, std::max(n_iters, 1));
    return esb * ((size_t)n_ck + (size_t)seg_len + 6) + grad_partials_bytes(g) + grad_block_partials_bytes(g) +
           (grad_keeps_steps(g, n_iters, ckpt_every) ? (size_t)seg_len * grad_step_bytes(g) : 0);
}

// Enqueues the whole gradient on s, with its work buffers at mem.
static pgm_status enqueue_grad(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                               int32_t n_iters, int32_t ckpt_every, const float *d_beliefs, float *d_log_pot,
                               float *d_evidence, char *mem, cudaStream_t s) {
    const int64_t ES = std::max<int64_t>(g->info.n_edge_states, 1);
    const size_t esb = align_up((size_t)ES * sizeof(float), 256);
    const int n_ck = n_iters > 0 ? (n_iters + ckpt_every - 1) / ckpt_every : 0;
    const int seg_len = std::min(ckpt_every, std::max(n_iters, 1));
    auto buf = [&](size_t i) { return reinterpret_cast<float *>(mem + i * esb); };
    float *ck = buf(0), *rec = buf(n_ck), *mA = buf(n_ck + seg_len), *mB = buf(n_ck + seg_len + 1);
    float *adjA = buf(n_ck + seg_len + 2), *adjB = buf(n_ck + seg_len + 3), *dv = buf(n_ck + seg_len + 4);
    float *ddamp = buf(n_ck + seg_len + 5);
    float *partials = g->adj_nc_max > 0 ? buf(n_ck + seg_len + 6) : nullptr;
    auto ckp = [&](int i) { return ck + (size_t)i * (esb / sizeof(float)); };
    auto recp = [&](int i) { return rec + (size_t)i * (esb / sizeof(float)); };
    // kept variable-pass outputs of the segment's iterations: step i's graph view points its
    // high-degree totals and belief residuals at the step's own buffers
    const bool keep = grad_keeps_steps(g, n_iters, ckpt_every);
    float *bpartials = grad_block_partials_bytes(g)
                           ? reinterpret_cast<float *>(mem + esb * ((size_t)n_ck + (size_t)seg_len + 6) +
                                                       grad_partials_bytes(g))
                           : nullptr;
    char *steps = mem + esb * ((size_t)n_ck + (size_t)seg_len + 6) + grad_partials_bytes(g) +
                  grad_block_partials_bytes(g);
    const size_t vsb = align_up((size_t)std::max<int64_t>(g->info.n_var_states, 1) * sizeof(float), 256);
    auto step_b = [&](int i) { return reinterpret_cast<float *>(steps + (size_t)i * grad_step_bytes(g)); };
    auto step_G = [&](int i) {
        DevGraph Gs = g->G;
        char *p = steps + (size_t)i * grad_step_bytes(g) + vsb;
        if (Gs.hd_b) {
            Gs.hd_b = reinterpret_cast<float *>(p);
            p += 4 * vsb;
        }
        if (Gs.b_lo) Gs.b_lo = reinterpret_cast<float *>(p);
        return Gs;
    };
    pgm_status st = PGM_OK;
    cudaError_t e = cudaSuccess;
    if (g->info.n_potentials > 0) e = cudaMemsetAsync(d_log_pot, 0, (size_t)g->info.n_potentials * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(mA, 0, esb, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(grad)");
    // forward with a checkpoint every ckpt_every iterations
    for (int t = 0; t < n_iters && st == PGM_OK; ++t) {
        if (t % ckpt_every == 0) {
            e = cudaMemcpyAsync(ckp(t / ckpt_every), mA, esb, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "checkpoint copy");
        }
        if (st == PGM_OK) st = one_iteration(g, log_pot, evidence, T, damping, mA, mB, s);
        std::swap(mA, mB);
    }
    // the belief read-out in reverse
    if (st == PGM_OK) {
        e = launch_adj_beliefs(g->G, evidence, mA, d_beliefs, d_evidence, adjA, s);
        if (e != cudaSuccess) st = cuda_fail(e, "adjoint beliefs launch");
    }
    // segments in reverse: recompute the states from the checkpoint, then step back
    for (int sgi = n_ck - 1; sgi >= 0 && st == PGM_OK; --sgi) {
        const int t0 = sgi * ckpt_every, t1 = std::min(t0 + ckpt_every, (int)n_iters);
        e = cudaMemcpyAsync(recp(0), ckp(sgi), esb, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = cuda_fail(e, "recompute copy");
        if (keep) {
            // each recomputed iteration's variable pass writes into its step's buffers,
            // which its reverse step reads; the segment's last state needs one more pass
            for (int i = 1; i <= t1 - t0 && st == PGM_OK; ++i) {
                const DevGraph Gs = step_G(i - 1);
                e = launch_var_pass(Gs, g->P, evidence, recp(i - 1), step_b(i - 1), kVarIter, nullptr, s);
                if (e == cudaSuccess && i < t1 - t0)
                    e = launch_factor_pass(Gs, g->P, log_pot, step_b(i - 1), evidence, recp(i - 1), recp(i), T,
                                           damping, s);
                if (e != cudaSuccess) st = cuda_fail(e, "recompute launch");
            }
        } else {
            for (int i = 1; i < t1 - t0 && st == PGM_OK; ++i)
                st = one_iteration(g, log_pot, evidence, T, damping, recp(i - 1), recp(i), s);
        }
        for (int t = t1; t > t0 && st == PGM_OK; --t) {
            const float *m_prev = recp(t - 1 - t0);
            const DevGraph Gs = keep ? step_G(t - 1 - t0) : g->G;
            float *bt = keep ? step_b(t - 1 - t0) : g->b;
            e = keep ? cudaSuccess : launch_var_pass(Gs, g->P, evidence, m_prev, bt, kVarIter, nullptr, s);
            if (e == cudaSuccess)
                e = launch_adj_factor(Gs, g->adj_launch, log_pot, bt, evidence, m_prev, adjA, dv, ddamp, d_log_pot,
                                      partials, g->adj_nc_max, T, damping, s);
            if (e == cudaSuccess)
                e = launch_adj_factor(Gs, g->adj_block_launch, log_pot, bt, evidence, m_prev, adjA, dv, ddamp,
                                      d_log_pot, bpartials, g->adj_block_nc_max, T, damping, s);
            if (e == cudaSuccess)
                e = launch_adj_logic(Gs, g->adj_logic_launch, bt, evidence, m_prev, adjA, dv, ddamp, T, damping, s);
            if (e == cudaSuccess) e = launch_adj_var(Gs, ddamp, dv, adjB, d_evidence, s);
            if (e != cudaSuccess) st = cuda_fail(e, "adjoint step launch");
            std::swap(adjA, adjB);
        }
    }
    return st;
}

static void drop_cached_grads(pgm_graph *g) {
    for (auto &c : g->grads) cudaGraphExecDestroy(c.exec);
    g->grads.clear();
}

pgm_status pgm_grad(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                    int32_t n_iters, int32_t ckpt_every, const float *d_beliefs, float *d_log_pot,
                    float *d_evidence, void *stream) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    if (!(T > 0.f) || !std::isfinite(T))
        return fail(T == 0.f ? PGM_ENOTSUP : PGM_EINVAL, "pgm_grad needs a finite T > 0 (max-product has no gradient)");
    if (!(damping >= 0.f && damping < 1.f)) return fail(PGM_EINVAL, "damping must be in [0, 1)");
    if (n_iters < 0 || ckpt_every < 1) return fail(PGM_EINVAL, "n_iters >= 0 and ckpt_every >= 1 required");
    if (!evidence || !d_beliefs || !d_evidence || (g->info.n_potentials > 0 && (!log_pot || !d_log_pot)))
        return fail(PGM_EINVAL, "NULL argument");
    if (g->has_xor) return fail(PGM_ENOTSUP, "pgm_grad: XOR factors have no adjoint in this build");
    if (pgm_status st = checked_gate(g, stream); st != PGM_OK) return st;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t total = grad_work_bytes(g, n_iters, ckpt_every);
    if (!g->use_cuda_graph || g->ordered) {  // stream-ordered work buffers, direct launches
        char *mem = nullptr;
        cudaError_t e = cudaMallocAsync(&mem, total, s);
        if (e != cudaSuccess) return fail(PGM_ENOMEM, std::string("cudaMallocAsync(grad): ") + cudaGetErrorString(e));
        pgm_status st = enqueue_grad(g, log_pot, evidence, T, damping, n_iters, ckpt_every, d_beliefs, d_log_pot,
                                     d_evidence, mem, s);
        cudaFreeAsync(mem, s);
        return st;
    }
    // CUDA graph of the whole call on persistent work buffers (grown when needed)
    if (g->grad_bytes < total) {
        cudaError_t e = cudaDeviceSynchronize();  // the old buffers may be in use by a replay
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
        drop_cached_grads(g);
        if (g->grad_mem) cudaFree(g->grad_mem);
        g->grad_mem = nullptr;
        g->grad_bytes = 0;
        if (cudaMalloc(&g->grad_mem, total) != cudaSuccess) {
            g->grad_mem = nullptr;
            return fail(PGM_ENOMEM, "cudaMalloc(grad)");
        }
        g->grad_bytes = total;
    }
    uint32_t tb, db;
    std::memcpy(&tb, &T, sizeof tb);
    std::memcpy(&db, &damping, sizeof db);
    cudaGraphExec_t exec = nullptr;
    for (auto &c : g->grads)
        if (c.log_pot == log_pot && c.evidence == evidence && c.d_beliefs == d_beliefs && c.d_log_pot == d_log_pot &&
            c.d_evidence == d_evidence && c.T_bits == tb && c.damping_bits == db && c.n_iters == n_iters &&
            c.ckpt_every == ckpt_every)
            exec = c.exec;
    if (!exec) {
        if (!g->capture_stream) {
            cudaError_t e = cudaStreamCreateWithFlags(&g->capture_stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        }
        cudaError_t e = cudaStreamBeginCapture(g->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        pgm_status st = enqueue_grad(g, log_pot, evidence, T, damping, n_iters, ckpt_every, d_beliefs, d_log_pot,
                                     d_evidence, static_cast<char *>(g->grad_mem), g->capture_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(g->capture_stream, &graph);
        if (st != PGM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (g->grads.size() >= 4) {
            cudaGraphExecDestroy(g->grads.front().exec);
            g->grads.erase(g->grads.begin());
        }
        g->grads.push_back({log_pot, evidence, d_beliefs, d_log_pot, d_evidence, tb, db, n_iters, ckpt_every, exec});
    }
    cudaError_t e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return PGM_OK;
}

pgm_status pgm_set_option(pgm_graph *g, int32_t option, int64_t value) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    switch (option) {
        case PGM_OPT_CUDA_GRAPH:
            g->use_cuda_graph = value != 0;
            if (!g->use_cuda_graph) drop_cached_runs(g);
            return PGM_OK;
        case PGM_OPT_LOG_RATIO:
            if (value < 0 || value > INT32_MAX) return fail(PGM_EINVAL, "PGM_OPT_LOG_RATIO must be >= 0");
            if (value != g->log_ratio_min_iters) drop_cached_runs(g);
            g->log_ratio_min_iters = (int32_t)value;
            return PGM_OK;
        case PGM_OPT_SMALL_RUN:
            if (value < 0 || value > 2) return fail(PGM_EINVAL, "PGM_OPT_SMALL_RUN must be 0, 1 or 2");
            if (value != g->small_run) drop_cached_runs(g);
            g->small_run = (int32_t)value;
            return PGM_OK;
        case PGM_OPT_ENUM_BLOCK: {
            if (value != 0 && value != 1) return fail(PGM_EINVAL, "PGM_OPT_ENUM_BLOCK must be 0 or 1");
            DeviceGuard dg(g->device);
            cudaError_t e = cudaDeviceSynchronize();  // a replay may be reading the segments
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            drop_cached_runs(g);
            for (size_t li = 0; li < g->P.factor.size(); ++li) {
                FactorLaunch &L = g->P.factor[li];
                if (L.base_variant != kEnumGeneric) continue;
                const int want = value ? kEnumBlock : kEnumGeneric;
                if (L.variant == want) continue;
                const int old_variant = L.variant;
                L.variant = want;
                if (!replan_factor_launch(g, li, want == kEnumBlock ? 256 : 128, nullptr)) {
                    L.variant = old_variant;
                    return fail(PGM_ECUDA, "re-planning an enumeration launch failed");
                }
            }
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            g->enum_block = (int32_t)value;
            return PGM_OK;
        }
        case PGM_OPT_CHECKED:
            if (value != 0 && value != 1) return fail(PGM_EINVAL, "PGM_OPT_CHECKED must be 0 or 1");
            g->checked = (int32_t)value;
            return PGM_OK;
        case PGM_OPT_PAIR_FORM: {
            if (value < 0 || value > 4) return fail(PGM_EINVAL, "PGM_OPT_PAIR_FORM must be 0..4");
            DeviceGuard dg(g->device);
            cudaError_t e = cudaDeviceSynchronize();  // a replay may be reading the segments
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            drop_cached_runs(g);
            for (size_t li = 0; li < g->P.factor.size(); ++li) {
                FactorLaunch &L = g->P.factor[li];
                const int base = L.base_variant;
                int K = 0;
                if (base == kPairT4 || base == kPair4 || base == kPairD4) K = 4;
                else if (base == kPairT8 || base == kPairQ8 || base == kPair8 || base == kPairD8) K = 8;
                else if (base == kPairT16 || base == kPairQ16 || base == kPair16 || base == kPairD16) K = 16;
                if (K == 0) continue;
                const int thr = K == 4 ? kPairT4 : K == 8 ? kPairT8 : kPairT16;
                const int lanes = K == 4 ? kPair4 : K == 8 ? kPair8 : kPair16;
                const int quad = K == 8 ? kPairQ8 : K == 16 ? kPairQ16 : thr;
                const int dir = K == 4 ? kPairD4 : K == 8 ? kPairD8 : kPairD16;
                // the K / 4-lane form runs launches whose groups all share their tables
                bool all_shared = true;
                const EnumSeg *sg = reinterpret_cast<const EnumSeg *>(g->factor_segs_host[li].data());
                for (int i = 0; i < L.n_seg; ++i) all_shared = all_shared && sg[i].shared != 0;
                const int want = value == 0 ? base : value == 1 ? thr : value == 2 ? lanes
                                 : value == 3 ? (all_shared ? quad : thr) : dir;
                if (L.variant == want) continue;
                const int old_variant = L.variant;
                L.variant = want;
                if (!replan_factor_launch(g, li, want == kPairT16 ? 128 : 256, nullptr)) {
                    L.variant = old_variant;
                    return fail(PGM_ECUDA, "re-planning a pairwise launch failed");
                }
            }
            e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
            g->pair_form = (int32_t)value;
            return PGM_OK;
        }
        default:
            return fail(PGM_EINVAL, "unknown option");
    }
}

pgm_status pgm_get_option(const pgm_graph *g, int32_t option, int64_t *value) {
    if (!g || !value) return fail(PGM_EINVAL, "NULL argument");
    switch (option) {
        case PGM_OPT_CUDA_GRAPH:
            *value = g->use_cuda_graph != 0;
            return PGM_OK;
        case PGM_OPT_LOG_RATIO:
            *value = g->P.lr ? g->log_ratio_min_iters : 0;
            return PGM_OK;
        case PGM_OPT_ENUM_BLOCK:
            *value = g->enum_block;
            return PGM_OK;
        case PGM_OPT_PAIR_FORM:
            *value = g->pair_form;
            return PGM_OK;
        case PGM_OPT_CHECKED:
            *value = g->checked;
            return PGM_OK;
        case PGM_OPT_SMALL_RUN: {
            DeviceGuard dg(g->device);  // whether the device can place the cluster form
            *value = small_run_used(g) ? g->small_run : 0;
            return PGM_OK;
        }
        default:
            return fail(PGM_EINVAL, "unknown option");
    }
}

pgm_status pgm_beliefs(pgm_graph *g, const float *evidence, const float *msgs, float *out,
                       int32_t normalise, void *stream) {
    if (!g || !evidence || !out) return fail(PGM_EINVAL, "NULL argument");
    if (!msgs && g->info.n_edge_states > 0) return fail(PGM_EINVAL, "msgs is NULL");
    if (pgm_status st = checked_gate(g, stream); st != PGM_OK) return st;
    DeviceGuard dg(g->device);
    cudaError_t e = launch_var_pass(g->G, g->P, evidence, msgs, out,
                                    normalise ? kVarNormalised : kVarBeliefs, nullptr,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "belief pass launch");
    return PGM_OK;
}

pgm_status pgm_decode(pgm_graph *g, const float *evidence, const float *msgs, int32_t *out,
                      void *stream) {
    if (!g || !evidence || !out) return fail(PGM_EINVAL, "NULL argument");
    if (!msgs && g->info.n_edge_states > 0) return fail(PGM_EINVAL, "msgs is NULL");
    if (pgm_status st = checked_gate(g, stream); st != PGM_OK) return st;
    DeviceGuard dg(g->device);
    cudaError_t e = launch_var_pass(g->G, g->P, evidence, msgs, nullptr, kVarDecode, out,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "decode pass launch");
    return PGM_OK;
}

pgm_status pgm_infer_host(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                          float damping, int32_t n_iters, float *beliefs, int32_t *decode,
                          void *stream) {
    if (!g || !evidence) return fail(PGM_EINVAL, "NULL argument");
    if (!log_pot && g->info.n_potentials > 0) return fail(PGM_EINVAL, "log_pot is NULL");
    if (pgm_status st = checked_gate(g, stream); st != PGM_OK) return st;
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const pgm_info &I = g->info;
    size_t b_pot = align_up(std::max<int64_t>(I.n_potentials, 1) * sizeof(float), 256);
    size_t b_ev = align_up(I.n_var_states * sizeof(float), 256);
    size_t b_msgs = align_up(std::max<int64_t>(I.n_edge_states, 1) * sizeof(float), 256);
    size_t b_dec = align_up(I.n_vars * sizeof(int32_t), 256);
    if (!g->host_io_mem) {
        char *m = nullptr;
        cudaError_t e = cudaMalloc(&m, b_pot + 2 * b_ev + b_msgs + b_dec);
        if (e != cudaSuccess) return fail(PGM_ENOMEM, std::string("cudaMalloc(io): ") + cudaGetErrorString(e));
        g->host_io_mem = m;
        g->io_pot = reinterpret_cast<float *>(m);
        g->io_ev = reinterpret_cast<float *>(m + b_pot);
        g->io_bel = reinterpret_cast<float *>(m + b_pot + b_ev);
        g->io_msgs = reinterpret_cast<float *>(m + b_pot + 2 * b_ev);
        g->io_dec = reinterpret_cast<int32_t *>(m + b_pot + 2 * b_ev + b_msgs);
    }
    cudaError_t e = cudaSuccess;
    if (I.n_potentials > 0)
        e = cudaMemcpyAsync(g->io_pot, log_pot, I.n_potentials * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->io_ev, evidence, I.n_var_states * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && I.n_edge_states > 0)
        e = cudaMemsetAsync(g->io_msgs, 0, I.n_edge_states * sizeof(float), s);
    if (e != cudaSuccess) return cuda_fail(e, "pgm_infer_host upload");
    pgm_status st = pgm_run_bp(g, g->io_pot, g->io_ev, T, damping, n_iters, g->io_msgs, stream);
    if (st != PGM_OK) return st;
    if (beliefs) {
        st = pgm_beliefs(g, g->io_ev, g->io_msgs, g->io_bel, 1, stream);
        if (st != PGM_OK) return st;
        e = cudaMemcpyAsync(beliefs, g->io_bel, I.n_var_states * sizeof(float), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "pgm_infer_host download");
    }
    if (decode) {
        st = pgm_decode(g, g->io_ev, g->io_msgs, g->io_dec, stream);
        if (st != PGM_OK) return st;
        e = cudaMemcpyAsync(decode, g->io_dec, I.n_vars * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "pgm_infer_host download");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return PGM_OK;
}

pgm_status pgm_set_profiling(pgm_graph *g, int32_t period) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    if (period < 0) return fail(PGM_EINVAL, "period must be >= 0");
    g->profiling = period;
    return PGM_OK;
}

// Moves every recorded sampled iteration (cached-graph replays and direct launches) into
// the per-launch totals.
static pgm_status collect_all_times(pgm_graph *g) {
    for (auto &r : g->runs) {
        pgm_status st = collect_run_times(g, r);
        if (st != PGM_OK) return st;
    }
    pgm_status st = accumulate_groups(g, g->events, g->prof_groups);
    g->prof_groups.clear();
    g->events_used = 0;
    return st;
}

static void reset_times(pgm_graph *g) {
    g->launch_ms.clear();
    g->launch_n.clear();
    g->graph_var_ms = g->graph_factor_ms = 0.0;
    g->prof_var_launches = g->prof_factor_launches = 0;
}

pgm_status pgm_pass_times(pgm_graph *g, double *var_ms, double *factor_ms, int64_t *n_var,
                          int64_t *n_factor) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
    pgm_status st = collect_all_times(g);
    if (st != PGM_OK) return st;
    if (var_ms) *var_ms = g->graph_var_ms;
    if (factor_ms) *factor_ms = g->graph_factor_ms;
    if (n_var) *n_var = g->prof_var_launches;
    if (n_factor) *n_factor = g->prof_factor_launches;
    reset_times(g);
    return PGM_OK;
}

pgm_status pgm_launch_times(pgm_graph *g, int32_t n, double *ms, int64_t *count, int32_t *n_positions) {
    if (!g || n < 0 || (n > 0 && (!ms || !count))) return fail(PGM_EINVAL, "NULL argument or n < 0");
    DeviceGuard dg(g->device);
    pgm_status st = collect_all_times(g);
    if (st != PGM_OK) return st;
    const int np = (int)g->launch_ms.size();
    for (int i = 0; i < n; ++i) {
        ms[i] = i < np ? g->launch_ms[i] : 0.0;
        count[i] = i < np ? g->launch_n[i] : 0;
    }
    if (n_positions) *n_positions = np;
    reset_times(g);
    return PGM_OK;
}

pgm_status pgm_checked_report(const pgm_graph *g, int32_t *array, int64_t *position, int64_t *value) {
    if (!g || !array || !position || !value) return fail(PGM_EINVAL, "NULL argument");
    *array = g->bad_array;
    *position = g->bad_pos;
    *value = g->bad_array >= 0 ? g->bad_value : 0;
    return PGM_OK;
}

pgm_status pgm_audit_desc(const pgm_graph_desc *desc, int32_t corrupt_array, int64_t corrupt_pos,
                          int64_t corrupt_value, int32_t *bad_array, int64_t *bad_pos) {
    g_last_error.clear();
    if (!bad_array || !bad_pos) return fail(PGM_EINVAL, "NULL argument");
    HostLayout H;
    const void *one = desc;
    std::string err = compile_graph(&one, 1, &H);
    if (!err.empty()) return fail(PGM_EINVAL, err);
    std::vector<int32_t> lr = lr_eligible(H) ? lr_slot_map(H) : std::vector<int32_t>{};
    std::vector<EnumSeg> esegs;
    std::vector<LogicSeg> lsegs;
    for (const HostEnumGroup &hg : H.enum_groups) esegs.push_back(hg.seg);
    for (const HostLogicGroup &hg : H.logic_groups) lsegs.push_back(hg.seg);
    std::vector<std::vector<int32_t>> lists;
    for (int k = 0; k < kNumVarKinds; ++k)
        if (!H.var_bucket[k].empty() && !H.var_bucket_identity[k]) lists.push_back(H.var_bucket[k]);
    // the test's corruption of one entry (corrupt_array < 0: none)
    if (corrupt_array >= 0) {
        auto poke = [&](auto &vec, const char *name) -> pgm_status {
            if (corrupt_pos < 0 || corrupt_pos >= (int64_t)vec.size())
                return fail(PGM_EINVAL, std::string("corrupt_pos outside ") + name);
            vec[(size_t)corrupt_pos] = (typename std::decay_t<decltype(vec)>::value_type)corrupt_value;
            return PGM_OK;
        };
        pgm_status st = PGM_OK;
        switch (corrupt_array) {
            case kAuditVsOff: st = poke(H.vs_off, "vs_off"); break;
            case kAuditVinOff: st = poke(H.vin_off, "vin_off"); break;
            case kAuditVinEs: st = poke(H.vin_es, "vin_es"); break;
            case kAuditEdgeVs: st = poke(H.edge_vs, "edge_vs"); break;
            case kAuditEdgeVar: st = poke(H.edge_var, "edge_var"); break;
            case kAuditTab4: st = poke(H.vin_tab4, "vin_tab4"); break;
            case kAuditLrPos: st = poke(lr, "lr_pos"); break;
            case kAuditParOff: st = poke(H.paroff_pool, "paroff_pool"); break;
            case kAuditCfg: st = poke(H.cfg_pool, "cfg_pool"); break;
            case kAuditBs: st = poke(H.bs_pool, "bs_pool"); break;
            case kAuditEnumSeg:
                if (corrupt_pos < 0 || corrupt_pos >= (int64_t)esegs.size()) return fail(PGM_EINVAL, "no such record");
                esegs[(size_t)corrupt_pos].es_base = (int32_t)corrupt_value;
                break;
            case kAuditLogicSeg:
                if (corrupt_pos < 0 || corrupt_pos >= (int64_t)lsegs.size()) return fail(PGM_EINVAL, "no such record");
                lsegs[(size_t)corrupt_pos].paroff_base = (int32_t)corrupt_value;
                break;
            case kAuditVarList:
                if (lists.empty()) return fail(PGM_EINVAL, "the graph has no variable lists");
                st = poke(lists[0], "variable lists");
                break;
            default: return fail(PGM_EINVAL, "unknown array id");
        }
        if (st != PGM_OK) return st;
    }
    std::vector<AuditArray> flat;
    auto add = [&](const int32_t *p, int64_t n, int64_t lo, int64_t hi, int neg, int id) {
        if (n > 0) flat.push_back(AuditArray{p, n, lo, hi, neg, id});
    };
    add(H.vs_off.data(), H.V + 1, 0, H.VS + 1, false, kAuditVsOff);
    add(H.vin_off.data(), H.V + 1, 0, H.E + 1, false, kAuditVinOff);
    add(H.vin_es.data(), (int64_t)H.vin_es.size(), 0, H.ES, false, kAuditVinEs);
    add(H.edge_vs.data(), (int64_t)H.edge_vs.size(), 0, H.VS, 2, kAuditEdgeVs);
    add(H.edge_var.data(), (int64_t)H.edge_var.size(), 0, H.V, false, kAuditEdgeVar);
    add(H.vin_tab4.data(), (int64_t)H.vin_tab4.size(), 0, H.ES, true, kAuditTab4);
    add(lr.data(), (int64_t)lr.size(), 0, lr_slot_count(H), false, kAuditLrPos);
    add(H.paroff_pool.data(), (int64_t)H.paroff_pool.size(), 0, H.E + 1, false, kAuditParOff);
    for (const auto &l : lists) add(l.data(), (int64_t)l.size(), 0, H.V, false, kAuditVarList);
    const AuditSizes z{H.V, H.VS, H.E, H.ES, H.P, (int64_t)H.cfg_pool.size(), (int64_t)H.bs_pool.size(),
                       (int64_t)H.paroff_pool.size(), H.cfg_pool.data(), H.bs_pool.data(), H.paroff_pool.data()};
    audit_host(flat, esegs, lsegs, z, bad_array, bad_pos);
    return PGM_OK;
}

pgm_status pgm_device_flags(pgm_graph *g, uint32_t *flags, int32_t clear, void *stream) {
    if (!g || !flags) return fail(PGM_EINVAL, "NULL argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaMemcpy(flags, g->G.flags, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(flags)");
    if (clear) {
        e = cudaMemset(g->G.flags, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(flags)");
    }
    return PGM_OK;
}

}  // extern "C"
