// Internal layout of a compiled factor graph (host compiler <-> kernels).
//
// The flat layout follows PGMax's flat-array design (arXiv 2202.04110, Sec. 4):
// every factor-to-variable message lives in one 1-D array indexed by edge-state, and
// the compiler keeps the global indices of variable states and factor configurations.
// Only factor-to-variable messages are stored; variable-to-factor messages are
// recomputed each iteration from the beliefs (b_v - m_{f->v}).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgm.h"

namespace pgm {

constexpr int kMaxArity = 8;
constexpr int kMaxStateSum = 64;          // thread-per-factor enumeration kernels
constexpr int kEnumBlockStateSum = 2048;  // block-per-factor form (kMaxArity x kMaxStates)
constexpr int kEnumGenericMaxCfg = 256;   // longer configuration lists use the block form
constexpr int kEnumBlockThreads = 256;
constexpr int kEnumWarpStateSum = 256;  // block form: a warp per factor up to this state sum
constexpr int kEnumTableSmem = 160 * 1024;  // largest configuration table staged per block
constexpr int kMaxStates = 256;
constexpr int kVarBlockDegree = 64;  // variables with more factors use a block each
constexpr int kVarBlockThreads = 256;
constexpr int kVarItems = 8;                               // contiguous edges per thread
constexpr int kVarTile = kVarBlockThreads * kVarItems;     // edges per tile
constexpr int kVarMaxTiles = 256;                          // degree limit 524,288
constexpr int kLogicSmallFan = 4;    // logical groups up to this fan-in: thread per factor

// Factor-pass kernel variants.
enum FactorVariant : int32_t {
    kPair2 = 0,   // dense pairwise table, both variables with 2 states
    kPair4 = 1,
    kPair8 = 2,
    kPair16 = 3,
    kEnumGeneric = 4,  // any listed-configuration factor within the limits
    kLogicSmall = 5,   // OR / AND, fan-in <= kLogicSmallFan, thread per factor
    kLogicWarp = 6,    // OR / AND, any fan-in, warp per factor
    kPairT4 = 7,       // dense pairwise table, K = 4, 8, 16, thread per factor (the
    kPairT8 = 8,       // alternative to the K-lane form kPair4 / 8 / 16; the autotuner
    kPairT16 = 9,      // picks per launch)
    kEnumBlock = 10,   // listed-configuration factors with a state sum above kMaxStateSum or
                       // a list longer than kEnumGenericMaxCfg: a block per run of factors
    kPairQ8 = 11,      // dense pairwise table shared by the group, K = 8, 16: K / 4 lanes per
    kPairQ16 = 12,     // factor, four states each (an alternative the autotuner may pick)
    kPairD4 = 13,      // dense pairwise table, K = 4, 8, 16: a thread per factor and
    kPairD8 = 14,      // direction (a warp pair per 32 factors; an alternative the autotuner
    kPairD16 = 15,     // may pick)
    kNumFactorVariants = 16
};

// One enumeration group as seen by a launch. Edges of factor f are
// edge_base + f * arity + j; their edge-states start at es_base + f * es_per_fac + Koff[j].
struct EnumSeg {
    int32_t block_begin;  // first block of the launch that works on this group
    int32_t n_fac;
    int32_t edge_base;
    int32_t es_base;
    int32_t es_per_fac;
    int32_t pot_base;     // first log-potential of the group
    int32_t shared;       // 1: one table of n_cfg values for all factors
    int32_t n_cfg;
    int32_t arity;
    int32_t cfg_base;     // offset of the group's [n_cfg * arity] table in the uint8 pool
    int32_t K[kMaxArity];
    int32_t Koff[kMaxArity];
    // block form (kEnumBlock) only:
    int32_t bs_base;      // offset in DevGraph::bs_pool of the group's lists by output
                          // state: es_per_fac + 1 offsets, then arity * n_cfg config ids
                          // (for each neighbour j and state x, the configs with state x
                          // at j, ascending); -1 if the group has none
    int32_t fpb;          // factors per block (set by the planner)
    int32_t lanes;        // threads per output state (1, 2, .., 32)
    int32_t table_bytes;  // bytes of the table staged in shared memory (0: read in place)
    int32_t packed;       // 1: pairwise, list entries (c << 11) | (Koff[other] + state)
    int32_t ordered;      // 1: reduce each output's configurations in ascending order
    int32_t member;       // the batch member the group belongs to
    int32_t dense;        // 1: a dense pairwise table, K0 = K1, configuration c = x K1 + y
};

// One logical group as seen by a launch. Factor f owns edges
// edge_base + par_off[f] + f + (0..n-1 parents, n child); every edge has 2 states, so
// edge e's states are at es_base + 2 * (e - edge_base).
struct LogicSeg {
    int32_t block_begin;
    int32_t n_fac;
    int32_t kind;         // 0 OR, 1 AND, 2 XOR
    int32_t edge_base;
    int32_t es_base;
    int32_t paroff_base;  // offset of the group's par_off[n_fac + 1] in the pool
    int32_t max_fan;
    int32_t member;       // the batch member the group belongs to
};

// Device-side view of a graph's index arrays (all int32, device memory).
struct DevGraph {
    int32_t V, VS, E, ES;
    const int32_t *vs_off;   // [V + 1]  first state of each variable
    const int32_t *vin_off;  // [V + 1]  CSR: incoming edges of each variable
    const int32_t *vin_es;   // [E]      first edge-state of each incoming edge
    const int32_t *edge_vs;  // [E]      first variable-state of each edge's variable; for
                             // a high-degree variable's edges with the sign bit set
    const uint8_t *cfg_pool;
    const int32_t *paroff_pool;
    uint32_t *flags;         // device status word
    const int4 *vin_tab4;    // [V] when every variable is binary with <= 4 factors: the
                             // first edge-states of its incoming edges, ascending, padded
                             // with -1 (else null)
    float *hd_b;             // [4 * VS] per state of a high-degree variable: the
                             // float-float sum of its finite evidence and incoming entries
                             // and the count of -inf ones (hi, lo, count, 0), from which a
                             // factor forms an edge's exact leave-one-out value; null if
                             // there are none
    const int32_t *bs_pool;  // configuration lists by output state (EnumSeg::bs_base)
    const int32_t *edge_var; // [E] each edge's variable (graphs with such lists), else null
    int64_t s_es, s_vs, s_pot;  // multi-sample launches (gridDim.y samples): per-sample
                                // strides of messages, evidence and beliefs, and
                                // log-potentials (0 if shared); 0 for ordinary launches
    const int32_t *frozen;   // [n_members] batches: nonzero = the factor pass skips the
                             // member (per-member early exit; zero outside such runs);
                             // null for single graphs and until first needed
    float *b_lo;             // [VS] graphs with variables of the warp pass (K > 16) or
                             // logical factors: what the iteration's beliefs b lost to
                             // rounding (b + b_lo is the float-float value), written for
                             // every warp-pass variable and for every other variable with
                             // an incoming entry beyond kExactThreshold; else null
    const int32_t *lr_pos;   // [E] Plan::lr graphs: each edge's slot in the log-ratio
                             // arrays (k V + v with vin_tab4, else its CSR index); else null
    const float *mem_prm;    // [4 n_members] batch runs with parameters per member: each
                             // member's (T, 1 / T, damping, 0); null otherwise
    float4 *hd_tot;          // tile totals of the high-degree variables' states (float-float
                             // sum of the finite entries, count of -inf ones, 0),
                             // VarLaunch::tiles; null if there are none
    int32_t *hd_cnt;         // [high-degree variables] tile tickets of k_var_hd (zero
                             // between launches); null if there are none
};

struct FactorLaunch {
    int32_t variant;
    int32_t n_seg;
    const void *segs;  // device EnumSeg[] or LogicSeg[]
    int32_t n_blocks;
    int32_t threads;
    int32_t smem;      // dynamic shared memory bytes
    int32_t max_fan;   // logical warp launches: largest fan-in
    int32_t max_blocks;  // K-lane pairwise launches: physical blocks (each walks a range
                         // of the n_blocks chunks)
    int32_t base_variant;  // the variant the compiler chose (before options and autotuning)
};

// Variable-pass kernel variants (buckets of variables).
enum VarKind : int32_t {
    kVarGeneric = 0,  // thread per variable, any K
    kVarBlock = 1,    // block per variable, degree > kVarBlockDegree
    kVarBinary = 2,   // thread per binary variable (float2 loads)
    kVarGroup4 = 3,   // K / 4 lanes per variable (4 states each), K = 4, 8, 16
    kVarGroup8 = 4,
    kVarGroup16 = 5,
    kVarWarp = 6,     // warp per variable, K > 16 (pgm_launch_info reports 7)
    kNumVarKinds = 7
};

struct VarLaunch {
    int32_t kind;            // VarKind
    int32_t n;               // variables in the list
    const int32_t *list;     // device list, or nullptr for the identity 0..n-1
    int32_t n_blocks;
    int32_t threads;
    int32_t dense_binary;    // every variable of the graph is binary (state offset = 2 v)
    // kVarBlock: the variables' tiles of kVarTile edges (int4: position in
    // the list, tile, first DevGraph::hd_tot entry of the variable, its tile count)
    const int4 *tiles;
    int32_t n_tiles;
};

struct Plan {
    std::vector<FactorLaunch> factor;
    std::vector<VarLaunch> var;
    // Binary pairwise graph (every variable binary, every factor a kPair2 factor, no
    // high-degree variable): iterations may keep one log-ratio per edge.
    bool lr = false;
    int32_t lr_blocks = 1;  // persistent log-ratio factor pass: blocks of 256 (8 per SM)
};

// Host-side result of the graph compiler (compile.cpp).
struct HostEnumGroup {
    int32_t variant;
    EnumSeg seg;  // block_begin filled by the planner
};
struct HostLogicGroup {
    int32_t variant;
    LogicSeg seg;
};

// Offsets of one member of a batch (a single graph is a batch of one) in the flat
// arrays of the compiled graph.
struct HostMember {
    int64_t var_off, n_vars, vs_off, n_var_states, edge_off, n_edges, es_off, n_edge_states,
        pot_off, n_potentials;
};

struct HostLayout {
    int64_t V = 0, VS = 0, E = 0, ES = 0, F = 0, P = 0;
    int32_t max_states = 0, max_degree = 0;
    std::vector<int32_t> vs_off, vin_off, vin_es, edge_vs;
    std::vector<int32_t> edge_var;  // [E] when a group has lists by output state, else empty
    std::vector<uint8_t> cfg_pool;    // each group's table starts on a 16-byte boundary
    std::vector<int32_t> paroff_pool;
    std::vector<int32_t> bs_pool;     // each group's lists start on a 16-byte boundary
    std::vector<HostEnumGroup> enum_groups;
    std::vector<HostLogicGroup> logic_groups;
    std::vector<int32_t> var_bucket[kNumVarKinds];  // variables of each VarKind, ascending
    bool var_bucket_identity[kNumVarKinds] = {};     // bucket is 0..V-1
    bool all_binary = false;
    std::vector<int32_t> vin_tab4;  // [4 * V] (see DevGraph::vin_tab4), empty if unused
    std::vector<HostMember> members;
};

// Graphs that keep belief residuals (DevGraph::b_lo): those with variables of the warp
// pass (K > 16) and those with logical factors.
inline bool keeps_b_lo(const HostLayout &H) { return !H.var_bucket[kVarWarp].empty() || !H.logic_groups.empty(); }

// Compiles n_desc graph descriptions (const pgm_graph_desc*) into one graph whose flat
// arrays hold the members one after the other. Returns "" on success, else an error.
std::string compile_graph(const void *const *descs, int n_desc, HostLayout *out);

// Called by a pass launcher after each of its kernel launches (per-launch event timing).
struct LaunchHook {
    void (*after)(void *ctx);
    void *ctx;
};

// Kernel launchers (kernels.cu). Each returns cudaGetLastError() of its launches.
// (n_samples > 1: samples as the launches' y dimension, at the strides of G)
cudaError_t launch_var_pass(const DevGraph &G, const Plan &P, const float *ev, const float *m,
                            float *b, int mode, int32_t *decode, cudaStream_t s, int n_samples = 1,
                            const LaunchHook *hook = nullptr);
cudaError_t launch_factor_pass(const DevGraph &G, const Plan &P, const float *log_pot,
                               const float *b, const float *ev, const float *m_old,
                               float *m_new, float T, float damping, cudaStream_t s, int n_samples = 1,
                               const LaunchHook *hook = nullptr);
// Log-ratio iteration of a Plan::lr graph (kernels.cu): d the factor-to-variable
// messages, lam the variable-to-factor values, one log-ratio per edge in variable order
// (slots DevGraph::lr_pos; 4V of them with vin_tab4, else E); the factor pass updates d
// in place.
// On the 4-slot layout (vin_tab4) the variable pass writes each variable's float-float
// total Dv[V] (lam only for variables that need the explicit sums) and the factor pass
// forms lam from it; otherwise lam is written and read.
cudaError_t launch_lr_var_pass(const DevGraph &G, const Plan &P, const float *ev, const float *d, float2 *Dv,
                               float *lam, cudaStream_t s, const LaunchHook *hook = nullptr);
// Per run: each factor's table as the three differences the update depends on (prm[3F]).
cudaError_t launch_lr_params(const DevGraph &G, const Plan &P, const float *log_pot, float *prm, cudaStream_t s);
cudaError_t launch_lr_factor_pass(const DevGraph &G, const Plan &P, const float *log_pot, const float *prm,
                                  const float2 *Dv, const float *lam, float *d, float T, float damping,
                                  cudaStream_t s, const LaunchHook *hook = nullptr);
// Many samples of one 4-slot log-ratio graph (sample index innermost; Sp = S for
// per-sample potentials, else 1): per run, the transposed evidence ev_s[V S], packed
// messages d[4V S] and table differences prm[3 F Sp]; per iteration, the variable pass
// (Dv[V S], lam[4V S] for flagged variables) and the factor pass; at the end, unpack.
cudaError_t launch_ms_prepare(const DevGraph &G, const Plan &P, int S, int Sp, int64_t n_pot,
                              const float *log_pot, const float *ev, const float *msgs, float2 *ev_s, float *d,
                              float *prm, cudaStream_t s);
cudaError_t launch_ms_iteration(const DevGraph &G, const Plan &P, int S, int Sp, int64_t n_pot,
                                const float *log_pot, const float *prm, const float2 *ev_s, float *d, float2 *Dv,
                                float *lam, float T, float damping, cudaStream_t s);
cudaError_t launch_ms_unpack(const DevGraph &G, int S, const float *d, float *msgs, cudaStream_t s);
// *out (zeroed by the caller; a float as its bit pattern) = max(*out, max_i |a[i] - b[i]|).
cudaError_t launch_residual(int64_t n, const float *a, const float *b, unsigned *out, int n_sm, cudaStream_t s);
// Early-exit loop control (a kernel in a conditional while body): *done += n; continue
// while the residual bits in *res are above tol (or NaN) and *done < limit.
cudaError_t launch_until_control(cudaGraphConditionalHandle h, const unsigned *res, int *done, int n, int limit,
                                 float tol, cudaStream_t s);
// Per-member early exit of a batch (member edge-state ranges off[n_members + 1]):
// state reset; residuals of the members not frozen (res[m] = max(res[m], max |a - b|));
// loop control after a trip of n iterations (frozen members' words: 2 = frozen this
// trip, its messages to be copied to the other buffer; 1 = frozen); the copy.
cudaError_t launch_until_members_init(int32_t *frozen, unsigned *res, int32_t *iters, float *resid,
                                      const int32_t *off, int n_members, int *state, cudaStream_t s);
cudaError_t launch_residual_members(int64_t n, const float *a, const float *b, const int32_t *off, int n_members,
                                    const int32_t *frozen, unsigned *res, int n_sm, cudaStream_t s);
cudaError_t launch_until_control_members(cudaGraphConditionalHandle h, bool set_condition, unsigned *res,
                                         int32_t *frozen, int32_t *iters, float *resid, int n_members, int *state,
                                         int n, int limit, float tol, cudaStream_t s);
cudaError_t launch_freeze_copy(const int32_t *frozen, const int32_t *off, int n_members, const float *a, float *b,
                               int n_sm, cudaStream_t s);
// Batch runs with iteration counts per member: members whose count is `it` are frozen
// and their message ranges (off[n_members + 1]) copied from a to b.
cudaError_t launch_batch_freeze(const int32_t *n_iters, int it, int n_members, const int32_t *off, int32_t *frozen,
                                const float *a, float *b, int n_sm, cudaStream_t s);
// out[s VS + i] = ev[i] + noise[s VS + i] (perturb-and-max-product evidence).
cudaError_t launch_pmp_perturb(int64_t VS, int S, const float *ev, const float *noise, float *out, cudaStream_t s);
// Log-ratio pack (from the [2E] edge-state layout; unused slots 0) and unpack.
cudaError_t launch_lr_pack(const DevGraph &G, const float *m, float *d, cudaStream_t s);
cudaError_t launch_lr_unpack(const DevGraph &G, const float *d, float *m, cudaStream_t s);
// One block, or a cluster of blocks sharing their shared memories, runs a whole log-ratio
// run of a small graph (4-slot layout), msgs in and out: one block up to kLrSmallMaxV
// variables and kLrSmallMaxF factors (one variable and one factor per thread, or two
// factors above kLrSmallThreads of them; 24 V bytes of shared memory), a cluster of C blocks
// up to C times that (the same per block on its share). C is 16 where the device places a
// cluster of 16 such blocks (a non-portable size), else 8 where it places 8, else there is
// no cluster form (lr_cluster_size, asked once per device).
constexpr int kLrSmallThreads = 1024, kLrSmallMaxV = 1024, kLrSmallMaxF = 2048;
constexpr int kLrClusterMax = 16;
int lr_cluster_size();
// Setting 1 of PGM_OPT_SMALL_RUN: one block up to this many variables, the cluster above
// (the cluster's two barriers per iteration cost about 1.1 us per iteration on a GB300; one
// block was faster up to 24 x 24 grids, the cluster from 28 x 28).
constexpr int kLrBlockAutoV = 700;
inline bool lr_block_fits(int V, int F) { return V > 0 && V <= kLrSmallMaxV && F <= kLrSmallMaxF; }
inline bool lr_cluster_fits(int V, int F) {
    const int C = lr_cluster_size();
    return C > 0 && V > 0 && V <= C * kLrSmallMaxV && F <= C * kLrSmallMaxF;
}
cudaError_t launch_lr_small_run(const DevGraph &G, const Plan &P, const float *log_pot, const float *ev,
                                float *msgs, float *lam, float T, float damping, int n_iters, bool cluster,
                                cudaStream_t s);
// Adjoint launchers (kernels.cu).
cudaError_t launch_adj_beliefs(const DevGraph &G, const float *ev, const float *m, const float *gnb, float *d_ev,
                               float *adj, cudaStream_t s);
// (thread-per-factor launches: `partials` [warps of the launch x nc_max] receives the
// per-warp sums of shared-table gradients, reduced into d_pot in warp order; may be null
// when no group shares a table)
cudaError_t launch_adj_factor(const DevGraph &G, const FactorLaunch &L, const float *pot, const float *b,
                              const float *ev, const float *m_old, const float *adj, float *dv2f, float *ddamp,
                              float *d_pot, float *partials, int nc_max, float T, float damping, cudaStream_t s);
cudaError_t launch_adj_logic(const DevGraph &G, const FactorLaunch &L, const float *b, const float *ev,
                             const float *m_old, const float *adj, float *dv2f, float *ddamp, float T, float damping,
                             cudaStream_t s);
cudaError_t launch_adj_var(const DevGraph &G, const float *ddamp, const float *dv2f, float *adj_prev, float *d_ev,
                           cudaStream_t s);
// Resident blocks per SM of the block-form enumeration kernel for a launch shape.
int enum_block_resident(int threads, int smem);
// Configure kernel attributes (large dynamic shared memory) once per process/device.
cudaError_t prepare_kernels(int max_smem_bytes);

// Build a graph whose allocations, uploads and frees (pgm_free) are stream-ordered on
// `s`, with CUDA-graph replay off (used by the serving loop; capi.cu): from a description,
// or from a layout compile_graph made (the serving loop compiles each request once).
int32_t build_graph_on_stream(const pgm_graph_desc *desc, cudaStream_t s, pgm_graph **out);
int32_t build_layout_on_stream(const HostLayout &H, cudaStream_t s, pgm_graph **out);
// Device bytes a graph built from this layout holds (index arrays and scratch).
int64_t layout_device_bytes(const HostLayout &H);

// Records `msg` as the calling thread's last error (pgm_last_error) and returns `code`.
int32_t set_last_error(int32_t code, const std::string &msg);

// Variable-pass modes.
// kVarIter: the beliefs the factor pass reads during an iteration, shifted per
// variable so that its largest state is 0 (plus exact leave-one-out values for
// high-degree variables); kVarBeliefs: raw beliefs e + sum m.
enum VarMode : int { kVarBeliefs = 0, kVarNormalised = 1, kVarDecode = 2, kVarIter = 3 };

}  // namespace pgm
