/*
 * pgm.h -- C ABI of the GB300 loopy belief propagation engine.
 *
 * The engine runs log-space loopy belief propagation (LBP) over a flat factor graph,
 * the method of PGMax (arXiv 2202.04110): discrete variables with varying numbers of
 * states and factor graphs of arbitrary topology (Sec. 3, "Easy specification of
 * general factor graphs"), enumeration factors listed by their valid configurations
 * (Sec. 5.2), logical factors with message updates linear in the fan-in (Sec. 3),
 * parallel message updates with damping (Sec. 3, after Pretti 2005), all messages kept
 * in flat arrays updated by gather/scatter (Sec. 4, the flat-array implementation),
 * LBP as a pure function of explicit message state (Sec. 3,
 * Sec. 5.3), MAP decoding (Sec. 5.1).
 *
 * Conventions for every call:
 *  - Return value: PGM_OK (0) or a negative pgm_status. pgm_last_error() returns a
 *    thread-local message describing the last failure of the calling thread.
 *  - "host" pointers are read during the call only; the caller keeps ownership.
 *  - "device" pointers are CUDA global-memory pointers on the device the graph was
 *    built on, owned by the caller, and must stay valid until the work queued on
 *    `stream` has finished. All device work is asynchronous on `stream` (a
 *    cudaStream_t passed as void*; NULL is the legacy default stream).
 *  - Flat layouts:
 *      evidence / beliefs [n_var_states]: variable-major, K_v log-space values for
 *        variable v, in variable order.
 *      log_pot [n_potentials]: enumeration groups in order; a group with
 *        shared_potentials = 0 holds n_fac * n_cfg values (factor-major), a group with
 *        shared_potentials = 1 holds one table of n_cfg values used by all its factors.
 *      msgs [n_edge_states]: the factor-to-variable messages. Edges are enumerated
 *        group by group, enumeration groups first and logical groups after, factor by
 *        factor; an enumeration factor contributes its neighbours in order, a logical
 *        factor its parents in order and then its child. Each edge holds K_v
 *        log-space values of its variable.
 *  - Graph handles are not thread-safe: calls on one pgm_graph from several host
 *    threads must be serialised by the caller, and work on one graph queued on
 *    different streams must not overlap (the graph owns one scratch area).
 */
#ifndef PGM_H
#define PGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pgm_status;

#define PGM_OK 0
#define PGM_EINVAL (-1)    /* invalid argument or malformed graph */
#define PGM_ENOMEM (-2)    /* device or host allocation failed */
#define PGM_ECUDA (-3)     /* a CUDA runtime call failed */
#define PGM_ENOTSUP (-4)   /* valid but unsupported request */
#define PGM_EBUSY (-5)     /* not admitted now (serving) */
#define PGM_ETIMEDOUT (-6) /* a bounded wait ran out */

#define PGM_LOGIC_OR 0  /* child = OR(parents)  */
#define PGM_LOGIC_AND 1 /* child = AND(parents) */
#define PGM_LOGIC_XOR 2 /* child = XOR(parents): parents and child have even parity */

/* Bits of the device status word (pgm_device_flags). */
#define PGM_FLAG_CONTRADICTION 1u /* a message or belief had every state at -inf */
#define PGM_FLAG_NAN 2u           /* a NaN reached a belief */
#define PGM_FLAG_INDEX 4u         /* checked mode: an index array entry out of range (pgm_checked_report) */

/* Limits of this build (checked by pgm_build). */
#define PGM_MAX_STATES 256        /* states per variable */
#define PGM_MAX_ENUM_ARITY 8      /* neighbours of an enumeration factor */
#define PGM_MAX_ENUM_STATE_SUM 2048 /* sum of K over one enumeration factor's neighbours */
#define PGM_MAX_ENUM_LIST 1073741824 /* n_cfg * arity of one enumeration group */

typedef struct pgm_graph pgm_graph;

/*
 * Enumeration factors (Sec. 5.2: a factor given by the list of its valid configurations).
 * All factors of a group share arity, configuration list and the state counts of their
 * j-th neighbours. Configurations that are not listed have log-potential -inf.
 */
typedef struct {
    int32_t arity;             /* neighbours per factor, 1..PGM_MAX_ENUM_ARITY */
    int32_t n_cfg;             /* listed configurations, >= 1 */
    const int32_t *cfg;        /* host [n_cfg * arity]: state of neighbour j in config c */
    int32_t n_fac;             /* factors in the group, >= 0 */
    const int32_t *vars;       /* host [n_fac * arity]: neighbour j of factor f */
    int32_t shared_potentials; /* 0: n_fac * n_cfg log-potentials; 1: one n_cfg table */
} pgm_enum_group;

/*
 * Logical factors (Sec. 3: three kinds of logical factor whose updates are linear in the
 * fan-in; the paper names none of them, and OR, AND and XOR are the three built): child =
 * OP(parents) over binary variables, log-potential 0 on valid configurations and -inf
 * otherwise. A factor may have zero parents (OR and XOR of nothing are 0, AND of nothing
 * is 1). pgm_grad supports OR and AND groups only (PGM_ENOTSUP for a graph with XOR).
 */
typedef struct {
    int32_t kind;            /* PGM_LOGIC_OR, PGM_LOGIC_AND or PGM_LOGIC_XOR */
    int32_t n_fac;           /* factors in the group */
    const int32_t *par_off;  /* host [n_fac + 1], par_off[0] = 0, non-decreasing */
    const int32_t *parents;  /* host [par_off[n_fac]] */
    const int32_t *child;    /* host [n_fac] */
} pgm_logic_group;

typedef struct {
    int32_t n_vars;            /* >= 1 */
    const int32_t *num_states; /* host [n_vars], each in 1..PGM_MAX_STATES */
    int32_t n_enum_groups;
    const pgm_enum_group *enum_groups;
    int32_t n_logic_groups;
    const pgm_logic_group *logic_groups;
} pgm_graph_desc;

typedef struct {
    int64_t n_vars;
    int64_t n_var_states;  /* length of evidence / beliefs */
    int64_t n_factors;
    int64_t n_edges;
    int64_t n_edge_states; /* length of msgs */
    int64_t n_potentials;  /* length of log_pot */
    int32_t max_states;
    int32_t max_degree;    /* largest number of factors on one variable */
    int64_t device_bytes;  /* device memory held by the graph (indices + scratch) */
    int32_t launches_per_iter; /* kernel launches of one pgm_run_bp iteration */
    int32_t n_members;         /* graphs in the batch (1 for pgm_build) */
} pgm_info;

/* Where one member of a batch lives in the flat arrays of the batched graph. */
typedef struct {
    int64_t var_off, n_vars;               /* variables */
    int64_t vs_off, n_var_states;          /* evidence / beliefs */
    int64_t edge_off, n_edges;             /* edges */
    int64_t es_off, n_edge_states;         /* messages */
    int64_t pot_off, n_potentials;         /* log-potentials */
} pgm_member;

/*
 * Compile a factor graph (Sec. 4: flatten messages into 1-D arrays and keep the
 * global indices of variable states and factor configurations). Validates the
 * description, builds the flat index arrays on the host, copies them once to the
 * current CUDA device, and allocates the graph's scratch (one message buffer and one
 * belief buffer). Blocking. On success *out owns all of it until pgm_free.
 * Errors: PGM_EINVAL (state index >= K, variable out of range, non-binary variable in
 * a logical factor, a group whose j-th neighbours differ in state count, sizes beyond
 * int32 or the limits above), PGM_ENOMEM, PGM_ECUDA.
 */
pgm_status pgm_build(const pgm_graph_desc *desc, pgm_graph **out);

/*
 * Host-only: validate a description and report the sizes its compiled graph will have
 * (device_bytes = index arrays + scratch), without touching any GPU. Same errors as
 * pgm_build's validation.
 */
pgm_status pgm_check_desc(const pgm_graph_desc *desc, pgm_info *info);

/*
 * Batch of many graphs (Sec. 5.3: processing batches of models in parallel). Compiles n
 * descriptions into one graph whose flat arrays hold the members one after the other:
 * member i's variables, evidence, beliefs, edges, messages and log-potentials are
 * contiguous ranges (pgm_batch_member) laid out exactly as pgm_build lays out that
 * member alone, with its variable indices shifted. Every pass of pgm_run_bp on the
 * batch is one launch per kernel variant over all members, and a member's results are
 * those of the member alone (the per-factor and per-variable arithmetic does not depend
 * on the batch). Same errors as pgm_build, per description.
 */
pgm_status pgm_build_batch(const pgm_graph_desc *const *descs, int32_t n, pgm_graph **out);

/*
 * A batch (pgm_build_batch; a single graph is a batch of one) with its own T, damping
 * and iteration count for every member (Sec. 5.3 batches of models; each member as a
 * pgm_run_bp call of its own): T, damping, n_iters are host arrays [n_members]; member m
 * runs n_iters[m] iterations at T[m] and damping[m] from its messages in msgs (in/out,
 * warm starts as in pgm_run_bp). Every iteration is one variable pass and one factor
 * pass over all members still running -- two factor launches per kernel variant when
 * the batch mixes max-product (T = 0) with other members --, and a member leaves the
 * factor pass once its count is reached. A member's messages equal pgm_run_bp of that
 * member alone with its parameters and PGM_OPT_LOG_RATIO 0 (the edge-state iteration is
 * used throughout). Blocking. The first call allocates 20 n_members bytes and the
 * members' early-exit state of pgm_run_bp_until_members, kept until pgm_free.
 * Errors: PGM_EINVAL for NULL arrays or pointers, a T[m] negative or not finite, a
 * damping[m] outside [0, 1), an n_iters[m] < 0 (the message names the member).
 */
pgm_status pgm_run_bp_batch(pgm_graph *g, const float *log_pot, const float *evidence, const float *T,
                            const float *damping, const int32_t *n_iters, float *msgs, void *stream);

/* Offsets of member i (0 <= i < pgm_info.n_members) of a batch. */
pgm_status pgm_batch_member(const pgm_graph *g, int32_t i, pgm_member *m);

/* Release a graph and its device memory (synchronises its device). NULL is a no-op. */
void pgm_free(pgm_graph *g);

/* Sizes of a compiled graph. */
pgm_status pgm_graph_info(const pgm_graph *g, pgm_info *info);

/*
 * n_iters flooding LBP iterations (Sec. 3: parallel updates with damping).
 * Each iteration, from the current messages m:
 *   b_v = e_v + sum_f m_{f->v};  m_{v->f} = b_v - m_{f->v}          (variable side)
 *   mt_{f->i}(x) = LSE_T{ phi_f(c) + sum_{j != i} m_{j->f}(c_j) : c_i = x }
 *                                           (enumeration; closed forms for OR / AND)
 *   m_{f->i} <- norm( delta * m_{f->i} + (1 - delta) * norm(mt_{f->i}) )
 * where LSE_T(z) = T log sum exp(z / T) (T = 1 sum-product, T = 0 max-product) and
 * norm subtracts the maximum over the edge's states (an all -inf message becomes 0
 * and raises PGM_FLAG_CONTRADICTION).
 *   log_pot  device [n_potentials] (may be NULL when n_potentials = 0)
 *   evidence device [n_var_states]
 *   msgs     device [n_edge_states], in/out: zeros for a cold start, the previous
 *            result for a warm start (messages are explicit state, Sec. 3).
 * Errors: PGM_EINVAL (T < 0 or not finite, damping outside [0, 1), n_iters < 0, NULL
 * pointers), PGM_ECUDA.
 */
pgm_status pgm_run_bp(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                      float damping, int32_t n_iters, float *msgs, void *stream);

/*
 * Beliefs b_v = e_v + sum_f m_{f->v} (device out [n_var_states]). normalise = 1
 * writes the normalised log-beliefs b_v - LSE_1(b_v) (log-marginals for T = 1).
 * A variable whose beliefs are all -inf stays -inf and raises PGM_FLAG_CONTRADICTION.
 */
pgm_status pgm_beliefs(pgm_graph *g, const float *evidence, const float *msgs, float *out,
                       int32_t normalise, void *stream);

/*
 * MAP decode (Sec. 5.1): out[v] = argmax_x b_v(x), lowest state on exact ties
 * (device out [n_vars] int32).
 */
pgm_status pgm_decode(pgm_graph *g, const float *evidence, const float *msgs, int32_t *out,
                      void *stream);

/*
 * End-to-end inference from HOST buffers (the call of a user without device memory of
 * their own): copies log_pot [n_potentials] and evidence [n_var_states] from host
 * memory to graph-owned device buffers, runs n_iters iterations from zero messages
 * (pgm_run_bp), and copies the normalised log-beliefs [n_var_states] (if beliefs is
 * not NULL) and the MAP decode [n_vars] (if decode is not NULL) back to host memory.
 * Blocking: returns after the results are in host memory. Host buffers that are
 * page-locked (cudaHostAlloc / pinned) transfer faster. The device buffers are
 * allocated on the first call and kept until pgm_free.
 */
pgm_status pgm_infer_host(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                          float damping, int32_t n_iters, float *beliefs, int32_t *decode,
                          void *stream);

/*
 * Per-pass timing with CUDA events on the launching stream. period = N > 0 makes every
 * following pgm_run_bp record an event before and after the variable pass and the
 * factor pass of every N-th iteration (iterations N-1, 2N-1, ... of each call); period
 * = 0 turns it off. With PGM_OPT_CUDA_GRAPH on, the records are event nodes of the
 * call's CUDA graph (graphs are cached per period), so the times are those of the
 * replayed graph; launching a cached graph again first waits for its previous replay
 * if that replay's times have not been collected. pgm_pass_times synchronises,
 * returns the summed durations (milliseconds) and launch counts of the sampled passes
 * since the last reset, and resets them. Used by the benchmark to attribute time to
 * kernels; a sparse period keeps the timed run undisturbed.
 */
pgm_status pgm_set_profiling(pgm_graph *g, int32_t period);
pgm_status pgm_pass_times(pgm_graph *g, double *var_ms, double *factor_ms, int64_t *n_var,
                          int64_t *n_factor);
/*
 * The same sampled iterations, per launch: with profiling on, each sampled iteration
 * records an event before its first launch and one after each launch, so launch i of
 * the iteration (in the order of pgm_launch_info for edge-state iterations; for log-ratio
 * iterations the variable pass, then the factor pass) is timed from the end of launch
 * i - 1. ms[i] (host [n]) = the summed durations of launch position i, count[i] = how
 * many were sampled; *n_positions (may be NULL) = positions recorded. Synchronises and
 * resets the times like pgm_pass_times (the two calls share one set of totals).
 * PGM_EINVAL for a NULL graph, n < 0 or NULL arrays with n > 0.
 */
pgm_status pgm_launch_times(pgm_graph *g, int32_t n, double *ms, int64_t *count, int32_t *n_positions);

/*
 * Gradient (Sec. 5.3: LBP as part of an end-to-end differentiable system): the
 * vector-Jacobian product of the normalised log-beliefs after n_iters iterations from
 * zero messages (pgm_run_bp then pgm_beliefs(normalise = 1)) with the cotangent
 * d_beliefs [n_var_states], i.e. the gradient of L = sum(d_beliefs * (b - LSE_1(b)))
 * with respect to the log-potentials (d_log_pot [n_potentials]) and the evidence
 * (d_evidence [n_var_states]); both outputs are overwritten. Reverse mode through the
 * unrolled iterations: the forward keeps a checkpoint of the messages every ckpt_every
 * iterations and the reverse pass recomputes each segment from its checkpoint
 * (device scratch of (ceil(n_iters / ckpt_every) + min(ckpt_every, n_iters) + 6) x
 * n_edge_states floats). With PGM_OPT_CUDA_GRAPH on (default) the scratch is kept with
 * the graph (grown when a call needs more, which synchronises the device) and the whole
 * call is recorded as a CUDA graph on first use of an argument tuple (up to 4 kept) and
 * replayed on the caller's stream; with it off, the scratch is a stream-ordered
 * allocation freed before the call's work ends.
 * Every sum is taken in a fixed order, so repeated calls give the same bits: gradients of
 * log-potentials shared by a group of factors with a state sum up to 64 through warp
 * partials (each warp of 32 factors adds its contributions by a fixed shuffle tree, then
 * the warps' partials are added in order); in the block form (state sums above 64) each
 * variable-to-factor adjoint and each configuration's gradient is gathered by one thread
 * in list order, shared tables through per-team rows added in order. (A block-form
 * shared table whose rows would exceed 512 MiB of scratch falls back to atomic adds.)
 * Logical OR / AND factors are differentiated through their closed forms (linear in the
 * fan-in); a factor whose incoming log-odds include an infinite one (a hard constraint)
 * passes no gradient to its variable-to-factor values.
 * Errors: PGM_ENOTSUP for T = 0 (max-product is not differentiable); PGM_EINVAL for a
 * non-finite or negative T, damping outside [0, 1),
 * n_iters < 0, ckpt_every < 1, NULL pointers.
 */
pgm_status pgm_grad(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                    int32_t n_iters, int32_t ckpt_every, const float *d_beliefs, float *d_log_pot,
                    float *d_evidence, void *stream);

/*
 * Read (and, with clear = 1, reset) the graph's device status word, a set of
 * PGM_FLAG_* bits raised by kernels. Synchronises `stream` first.
 */
pgm_status pgm_device_flags(pgm_graph *g, uint32_t *flags, int32_t clear, void *stream);

/*
 * Checked mode: the first index-array violation found on this graph (*array = -1 if
 * none): the array (0 vs_off, 1 vin_off, 2 vin_es, 3 edge_vs, 4 edge_var, 5 vin_tab4,
 * 6 lr_pos, 7 paroff_pool, 8 cfg_pool, 9 configuration lists, 10 enumeration group
 * records, 11 logical group records, 12 variable lists), the entry's position (the
 * record's index for 10 and 11) and its value (-1 where none is read back). Host only.
 */
pgm_status pgm_checked_report(const pgm_graph *g, int32_t *array, int64_t *position, int64_t *value);

/*
 * Host only, no GPU: compiles a description and runs the checked-mode range checks on
 * the host copies of its index arrays (the same rules as the device checks), after
 * writing corrupt_value into entry corrupt_pos of array corrupt_array (ids as in
 * pgm_checked_report; for the records 10 / 11 the value replaces the record's first
 * edge-state / parent-offset base; for 12 the first variable list) when corrupt_array
 * >= 0. *bad_array, *bad_pos = the first violation in array order, -1 if none. For tests
 * of the checks on hosts without a GPU. PGM_EINVAL for a bad description or a corrupt
 * position outside the array.
 */
pgm_status pgm_audit_desc(const pgm_graph_desc *desc, int32_t corrupt_array, int64_t corrupt_pos,
                          int64_t corrupt_value, int32_t *bad_array, int64_t *bad_pos);

/*
 * Allocation-free LBP on a rows x cols grid of binary variables with one pairwise factor
 * per pair of 4-neighbours. The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory -- a process whose device memory is owned
 * and budgeted by a host framework, or code that must not call cudaMalloc / cudaFree
 * after start-up -- and so cannot use pgm_build / pgm_run_bp, which allocate the graph's
 * index arrays and scratch. It needs no graph object and allocates nothing: the grid
 * topology is computed from (row, column), and the scratch (the partner of `msgs` in the
 * ping-pong of iterations, the per-iteration beliefs, a status word) is one static
 * device array of PGM_NOALLOC_SCRATCH_FLOATS floats (16 MiB), which every GPU that loads
 * this library holds until the process exits.
 *   Layout (the graph pgm_build makes from the same grid with its factors listed cell by
 *   cell, row-major, each cell's right pair then its down pair): factor f has
 *   log_pot[4f .. 4f+3] over the configurations (0,0),(0,1),(1,0),(1,1) and messages
 *   msgs[4f .. 4f+1] (to the cell) and msgs[4f+2 .. 4f+3] (to the right or lower
 *   neighbour); evidence is [2 * rows * cols]. All pointers are device memory owned by
 *   the caller (log_pot and msgs 16-byte aligned, evidence 8-byte aligned); msgs is
 *   in/out as in pgm_run_bp, whose iteration this is.
 *   Limit: 4 * n_factors + 2 * rows * cols <= PGM_NOALLOC_SCRATCH_FLOATS, with
 *   n_factors = 2 * rows * cols - rows - cols (the largest square grid is 648 x 648);
 *   larger grids return PGM_EINVAL with the sizes in pgm_last_error().
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call before any
 *   stream capture. Every call on a device shares the one array, so calls whose work
 *   overlaps on the GPU (different streams, or different host threads) race and corrupt
 *   each other's results: serialise them. Each call clears the array's status word and
 *   then raises PGM_FLAG_CONTRADICTION in it when a message has both states at -inf (the
 *   message becomes 0, as in pgm_run_bp); pgm_grid2_noalloc_flags reads it.
 */
#define PGM_NOALLOC_SCRATCH_FLOATS 4194304
pgm_status pgm_grid2_run_bp_noalloc(int32_t rows, int32_t cols, const float *log_pot,
                                    const float *evidence, float T, float damping,
                                    int32_t n_iters, float *msgs, void *stream);
/*
 * The status word of the last pgm_grid2_run_bp_noalloc call on the current device (its
 * PGM_FLAG_* bits; 0 before any call): synchronises `stream`, copies the word into
 * *flags (host) and, with clear = 1, zeroes it. Allocates nothing. PGM_EINVAL for NULL
 * flags, PGM_ECUDA if the array's address cannot be looked up or a copy fails.
 */
pgm_status pgm_grid2_noalloc_flags(uint32_t *flags, int32_t clear, void *stream);

/*
 * n_samples runs of one graph with different inputs, as n_samples calls of pgm_run_bp:
 * sample s uses evidence[s * n_var_states ...], msgs[s * n_edge_states ...] (in/out,
 * the pgm_run_bp layout for each sample), and log_pot[s * n_potentials ...] if
 * pot_per_sample, else the one log_pot for every sample (Sec. 5.3 names batches of
 * samples processed in parallel as a use of the pure-function design). On a graph that takes log-ratio iterations
 * (PGM_OPT_LOG_RATIO) with at most 4 factors per variable, the samples run together in
 * chunks: one variable pass and one factor pass per iteration over a chunk's samples,
 * with the sample index innermost, so the graph's index arrays (and a shared table set)
 * are read once per iteration for the chunk; results equal those of the single-sample
 * runs. A chunk holds as many samples as keep the arrays exchanged between the passes
 * (about 32 bytes per variable and sample, plus 12 per factor and sample for
 * per-sample tables) within half the L2; where one sample alone exceeds that (e.g. a
 * 1000 x 1000 grid), the samples run one after another as pgm_run_bp. On every other
 * graph the samples run side by side as the second grid dimension of each edge-state
 * launch (one variable pass and one factor pass per iteration for a chunk, the index
 * arrays shared), in chunks whose per-sample scratch (a message buffer, beliefs, and the
 * graph's leave-one-out and residual buffers if it has them) stays within 1 GiB;
 * results equal those of the single-sample runs. The first call with a larger chunk
 * than before allocates device buffers, synchronising the device; they are kept until
 * pgm_free. Stream-ordered otherwise.
 * PGM_EINVAL for n_samples < 1 or the pgm_run_bp argument errors.
 */
pgm_status pgm_run_bp_multi(pgm_graph *g, int32_t n_samples, const float *log_pot, int32_t pot_per_sample,
                            const float *evidence, float T, float damping, int32_t n_iters, float *msgs,
                            void *stream);

/*
 * pgm_run_bp with an early exit: up to max_iters iterations in chunks of check_every;
 * the last iteration of each chunk is checked, residual = max over edge-states of
 * |m_t - m_{t-1}| (messages are max-normalised, so this is scale-free; equal infinite
 * entries count 0), and the run stops after the first chunk whose residual is <= tol.
 * *iters_done (may be NULL) = iterations run, *residual (may be NULL) = the last
 * residual checked (NaN if none was, i.e. max_iters = 0). The messages are those of
 * chunked pgm_run_bp calls (chunk - 1 iterations, then 1), so on a graph with
 * log-ratio iterations they can differ by rounding from one pgm_run_bp of the same
 * length. With PGM_OPT_CUDA_GRAPH on, the full chunks run as one CUDA graph whose
 * conditional while node repeats a chunk on the device while its residual is above tol
 * (recorded once per argument tuple, up to 4 kept): the call synchronises the stream
 * once, plus once for a last chunk shorter than check_every; with it off, after each
 * chunk. Blocking. The first call allocates an [n_edge_states] buffer and two pinned
 * words, kept until pgm_free. PGM_EINVAL for
 * check_every < 1, tol < 0 or NaN, or the pgm_run_bp argument errors.
 */
pgm_status pgm_run_bp_until(pgm_graph *g, const float *log_pot, const float *evidence, float T, float damping,
                            int32_t max_iters, float tol, int32_t check_every, float *msgs, int32_t *iters_done,
                            float *residual, void *stream);

/*
 * Perturb-and-max-product samples (the sampler of the binary-deconvolution example of
 * Sec. 5.2, after Lazaro-Gredilla et al. 2021): for each sample s, max-product (T = 0)
 * LBP for n_iters iterations from zero messages on the model whose evidence is
 * evidence + noise[s * n_var_states ...] (the caller draws the perturbations, e.g. Gumbel
 * noise), then the MAP decode of that model into samples[s * n_vars ...]. msgs
 * [n_samples * n_edge_states] is caller-owned working memory and holds each sample's
 * final messages on return. Runs the samples through pgm_run_bp_multi. The first call
 * with more samples than before allocates the perturbed-evidence buffer (n_samples *
 * n_var_states floats), synchronising the device; it is kept until pgm_free.
 * PGM_EINVAL for n_samples < 1, NULL noise / samples or the pgm_run_bp argument errors.
 */
pgm_status pgm_pmp_sample(pgm_graph *g, int32_t n_samples, const float *log_pot, const float *evidence,
                          const float *noise, float damping, int32_t n_iters, float *msgs, int32_t *samples,
                          void *stream);

/*
 * Early exit per member of a batch (pgm_build_batch; a single graph is a batch of one):
 * every member runs until the first checked iteration whose residual over its own
 * messages, max |m_t - m_{t-1}|, is <= tol (checked every check_every iterations), or
 * max_iters; from then on the factor pass skips the stopped member's factors and leaves
 * its messages at that iteration, while the other members go on. iters_done[m] and
 * residual[m] (host arrays [n_members]) are each member's iterations and last checked
 * residual (NaN before any check; 0 iterations and residual 0 for a member without
 * edges). A member's messages equal pgm_run_bp_until of that member alone with
 * PGM_OPT_LOG_RATIO 0: the run uses the edge-state iteration throughout. With
 * PGM_OPT_CUDA_GRAPH on, the full chunks run as one CUDA graph whose conditional while
 * node repeats a chunk while a member is active (recorded once per argument tuple, up to
 * 4 kept with those of pgm_run_bp_until); the rest is checked by the host. Blocking. The
 * first call allocates 4 (n_edge_states + 5 n_members) bytes, kept until pgm_free.
 * PGM_EINVAL for check_every < 1, tol < 0 or NaN, NULL outputs, and as pgm_run_bp.
 */
pgm_status pgm_run_bp_until_members(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                                    float damping, int32_t max_iters, float tol, int32_t check_every,
                                    float *msgs, int32_t *iters_done, float *residual, void *stream);

/*
 * Options of a graph. PGM_OPT_CUDA_GRAPH (default 1): pgm_run_bp with n_iters >= 2
 * (and per-pass profiling off) records the whole call -- every kernel of every
 * iteration and the final copy -- as a CUDA graph the first time it sees a given
 * (log_pot, evidence, msgs, T, damping, n_iters), on a private stream, and afterwards
 * replays it on the caller's stream (one launch per call; up to 8 cached per graph,
 * least recently used dropped). 0 launches the kernels one by one and drops the cache.
 * A cached graph holds the pointers it was recorded with: buffers that are freed and
 * reused at the same address with the same meaning are fine.
 */
#define PGM_OPT_CUDA_GRAPH 1
/*
 * PGM_OPT_LOG_RATIO (default 4; 0 = off): on a binary pairwise graph (every variable
 * binary, every factor a 2 x 2 enumeration factor, no variable with more than 64
 * factors), pgm_run_bp with n_iters >= the value keeps one number per edge and
 * direction during the iterations: the log-ratio d = m(1) - m(0) of each max-
 * normalised factor-to-variable message (the normalisation of Sec. 3 makes one entry
 * 0, so the encoding loses nothing) and of each variable-to-factor message, the latter
 * an exact leave-one-out sum rather than belief minus message. msgs is converted at
 * the start (messages that are not max-normalised are normalised, which the update
 * does not see) and written back in the [n_edge_states] layout at the end. The
 * iteration is the same; results differ from the option-off path by rounding only.
 * Negative values: PGM_EINVAL. pgm_launch_info / launches_per_iter do not count the 3
 * launches per run around the iterations (pack, table differences, unpack).
 */
#define PGM_OPT_LOG_RATIO 2
/*
 * PGM_OPT_ENUM_BLOCK (default 0): listed-configuration groups (factors that are not
 * dense pairwise tables) run with a thread per factor when their state sum is at most
 * 64 and their list at most 256 configurations, else with a block per run of factors
 * that stages the group's configuration table in shared memory. 1 moves the
 * thread-per-factor launch to the block form as well (0 moves it back), with one thread
 * per output state so that both give the same bits. Blocking (synchronises the device,
 * re-plans the launch, drops the cached CUDA graphs); values other than 0 and 1:
 * PGM_EINVAL.
 */
#define PGM_OPT_ENUM_BLOCK 3
/*
 * PGM_OPT_PAIR_FORM (default 0): the kernel form of dense K-state pairwise groups (K = 4,
 * 8, 16). 0 the compiler's choice (a thread per factor), 1 a thread per factor, 2 K
 * lanes per factor, 3 K / 4 lanes per factor with four states each (K = 8, 16, for
 * launches whose groups all share their tables; else a thread per factor), 4 a thread per
 * factor and direction. The thread, K / 4-lane and direction forms give the same bits.
 * Blocking like PGM_OPT_ENUM_BLOCK; pgm_autotune may change the forms afterwards.
 * Values outside 0..4: PGM_EINVAL.
 */
#define PGM_OPT_PAIR_FORM 4
/*
 * PGM_OPT_CHECKED (default 0): 1 turns on checked mode. Every call that launches kernels
 * on the graph (pgm_run_bp and the runs built on it, pgm_beliefs, pgm_decode, pgm_grad,
 * pgm_autotune, pgm_infer_host) first range-checks, on the device, every entry of the
 * graph's index arrays -- the per-variable state offsets and incoming-edge lists, each
 * edge's variable state, the padded incoming-edge table, the log-ratio slot map, the
 * logical groups' parent offsets, the configuration tables and lists by output state,
 * the group records of every launch and the variable lists of the variable pass --
 * against the range the kernels assume (these arrays are where every gathered index of
 * Sec. 4's flat layout comes from), and waits for the result. On a violation it raises
 * PGM_FLAG_INDEX in the status word (pgm_device_flags), keeps the array, position and
 * value for pgm_checked_report, and returns PGM_EINVAL without launching anything that
 * reads the arrays; nothing traps. The checks synchronise the stream on every call.
 * Values other than 0 and 1: PGM_EINVAL.
 */
#define PGM_OPT_CHECKED 5
/*
 * PGM_OPT_SMALL_RUN (default 1): a log-ratio run (PGM_OPT_LOG_RATIO) of a graph whose
 * variables have at most 4 factors each is one kernel launch: one thread block for at most
 * 700 variables (and 2,048 factors), else a cluster of C thread blocks on C SMs, whose
 * shared memories together hold the run's state, for at most 1,024 C variables and 2,048 C
 * factors: C = 16 where the device places a cluster of 16 such blocks (GB300: up to 16,384
 * variables), else 8 where it places 8, else no cluster form. 2 takes the cluster at every
 * size up to its limits. The launch converts msgs, runs
 * every iteration with the exchanged arrays in shared memory (24 bytes per variable) and a
 * block or cluster barrier after each pass, and writes msgs back, instead of 2 launches per
 * iteration plus 3. The arithmetic per variable and per factor is that of the multi-launch
 * iterations, so the messages and flags are bitwise the same. 0 turns it off. Per-pass
 * profiling (pgm_set_profiling) keeps the multi-launch form, which is also the one that
 * launches_per_iter and pgm_launch_info describe. Changing it drops the cached CUDA
 * graphs. pgm_get_option returns the setting where a log-ratio run of the graph takes
 * this form, else 0 (it asks the device once whether the cluster fits). Values outside
 * 0..2: PGM_EINVAL.
 */
#define PGM_OPT_SMALL_RUN 6
pgm_status pgm_set_option(pgm_graph *g, int32_t option, int64_t value);
/*
 * The option's effective value in *value: for PGM_OPT_CUDA_GRAPH, PGM_OPT_ENUM_BLOCK,
 * PGM_OPT_PAIR_FORM and PGM_OPT_CHECKED the setting; for PGM_OPT_LOG_RATIO the setting
 * if the graph qualifies, else 0; for PGM_OPT_SMALL_RUN the setting if it is on and the
 * graph qualifies, else 0. PGM_EINVAL for a NULL argument or an unknown option. No
 * device work (beyond one occupancy query per device for PGM_OPT_SMALL_RUN).
 */
pgm_status pgm_get_option(const pgm_graph *g, int32_t option, int64_t *value);

/*
 * Launch-shape autotuner: for every factor-pass launch of the graph (one per kernel
 * variant, covering all groups of that variant) times each thread-block shape the
 * kernel allows, and for dense K-state pairwise launches (K = 4, 8, 16) every kernel
 * form (K lanes per factor, thread per factor, and for shared tables K / 4 lanes per
 * factor), for listed-configuration launches both
 * forms (thread per factor, block per run of factors; the former only where every group
 * fits it) -- threads per block for the thread-per-factor kernels, warps per
 * block (factors per block) for the warp-per-factor logical kernel -- on the given
 * inputs, and keeps the fastest; likewise the block size of the thread-per-variable
 * pass. Allocates two temporary message buffers (freed before returning), blocks until
 * done, drops the cached CUDA graphs. Results are unchanged by the shapes.
 */
pgm_status pgm_autotune(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                        float damping, void *stream);

/*
 * Launch i of one iteration (0 <= i < pgm_info.launches_per_iter): kind 0 = variable
 * pass (variant 0 thread per variable, 1 variables with more than 64 factors: a block
 * per tile of 2048 incoming edges, the last tile of a variable finishing it; 2 thread
 * per binary variable, 3..5 K = 4, 8, 16 lanes per variable, 6 padded 4-edge table, 7
 * warp per variable with K > 16),
 * kind 1 = factor pass (variant: 0 dense pairwise K = 2; 1..3 dense pairwise K = 4, 8,
 * 16 with K lanes per factor; 4 listed configurations; 5 logical (OR / AND / XOR) thread
 * per factor; 6 logical warp per factor; 7..9 dense pairwise K = 4, 8, 16 with a thread
 * per factor, the default form, which pgm_autotune may exchange with 1..3, 11, 12 or
 * 13..15; 10 listed configurations with a block per run of factors; 11, 12 dense
 * pairwise K = 8, 16 with K / 4 lanes per factor, for shared tables; 13..15 dense
 * pairwise K = 4, 8, 16 with a thread per factor and direction); threads per block and
 * blocks. Any output pointer may be NULL.
 */
pgm_status pgm_launch_info(const pgm_graph *g, int32_t i, int32_t *kind, int32_t *variant,
                           int32_t *threads, int32_t *n_blocks);

/*
 * Serving loop: continuous admission of inference requests onto one GPU.
 * A request is a graph description with its log-potentials and evidence (host memory,
 * copied at submission), T, damping and an iteration count; its result is the
 * normalised log-beliefs and the MAP decode after n_iters iterations from zero messages
 * (pgm_run_bp + pgm_beliefs + pgm_decode). Requests queue in arrival order; up to
 * max_in_flight of them are on the GPU at once, each on its own stream. A free worker
 * takes the head of the queue and compiles its graph on the host (once; the workers
 * compile in parallel), and requests are admitted in arrival order, each as soon as its
 * device memory (compiled graph, scratch, inputs, outputs; stream-ordered allocations)
 * fits memory_budget_bytes together with the requests in flight. Kernels of in-flight
 * requests overlap on the device; a request's messages stay resident until it
 * finishes; max_in_flight = 1 runs one request at a time in arrival order. Results are
 * those of the same request run alone. Latency = submission to results in host memory.
 * The server's worker threads are its own; all calls are thread-safe.
 */
typedef struct pgm_server pgm_server;

typedef struct {
    int64_t memory_budget_bytes; /* device memory for requests in flight, > 0 */
    int32_t max_in_flight;       /* concurrent requests (worker threads and streams), 1..64 */
    int32_t max_pending;         /* queued requests before pgm_serve_submit returns PGM_EBUSY */
} pgm_server_config;

typedef struct {
    int64_t submitted, completed, failed, pending, in_flight;
    int64_t bytes_in_use, peak_bytes; /* device memory accounted to requests in flight */
    int64_t updates_done;             /* edge-state message updates of completed requests */
    double span_s;                    /* first submission to last completion, seconds */
    /* where completed requests spent their latency, seconds summed over them: in the
     * queue until a worker took them, compiling the graph on the host, waiting for
     * admission (their turn in arrival order and device memory), and on the device
     * (build and upload, iterations, read-back, free) */
    double queue_s, compile_s, admit_s, run_s;
} pgm_server_stats;

/* Create a server on the current device (starts max_in_flight worker threads). */
pgm_status pgm_serve_create(const pgm_server_config *cfg, pgm_server **out);

/*
 * Queue a request; *id identifies it. The description and host arrays are copied (they
 * may be freed on return); the graph is compiled and validated by the worker that
 * admits it (errors are reported by pgm_serve_poll / pgm_serve_wait). Never waits for
 * the GPU. Errors: PGM_EINVAL (argument checks), PGM_EBUSY (queue full).
 */
pgm_status pgm_serve_submit(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                            const float *evidence, float T, float damping, int32_t n_iters,
                            int64_t *id);

/*
 * pgm_serve_submit with an early exit: the request runs as pgm_run_bp_until (up to
 * max_iters iterations, stopping after the first checked iteration whose residual
 * max |m_t - m_{t-1}| is <= tol, checked every check_every iterations), so a request
 * that converges early frees its slot and memory early. Results equal pgm_run_bp_until
 * of the same request alone (the residual checks are host-side on the serving streams);
 * pgm_server_stats.updates_done counts the iterations actually run. Errors as
 * pgm_serve_submit, plus PGM_EINVAL for check_every < 1 or tol < 0 / NaN.
 */
pgm_status pgm_serve_submit_until(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                                  const float *evidence, float T, float damping, int32_t max_iters,
                                  float tol, int32_t check_every, int64_t *id);

/*
 * pgm_serve_submit (check_every = 0) or pgm_serve_submit_until (check_every >= 1, tol)
 * without copies: the description (with every array it points to), log_pot and
 * evidence are borrowed, and must stay valid and unchanged until pgm_serve_poll /
 * pgm_serve_wait has returned the request's result (or pgm_serve_destroy has
 * returned). For callers that submit many requests of a few graph structures at a
 * high rate (copying a large grid's description and evidence at every submission
 * bounds the submission rate). The description is validated by the worker that admits
 * the request (errors reported by pgm_serve_poll / pgm_serve_wait).
 */
pgm_status pgm_serve_submit_borrowed(pgm_server *s, const pgm_graph_desc *desc, const float *log_pot,
                                     const float *evidence, float T, float damping, int32_t max_iters,
                                     float tol, int32_t check_every, int64_t *id);

/*
 * Result of request `id`: PGM_EBUSY while it is queued or running; otherwise copies the
 * normalised log-beliefs [n_var_states] and decode [n_vars] into the host buffers (each
 * may be NULL), writes the latency in seconds, forgets the request and returns its
 * status (PGM_ENOMEM if it alone exceeds the memory budget, a build or CUDA error).
 */
pgm_status pgm_serve_poll(pgm_server *s, int64_t id, float *beliefs, int32_t *decode,
                          double *latency_s);

/* pgm_serve_poll that waits up to timeout_us microseconds; PGM_ETIMEDOUT if not done. */
pgm_status pgm_serve_wait(pgm_server *s, int64_t id, int64_t timeout_us, float *beliefs,
                          int32_t *decode, double *latency_s);

pgm_status pgm_serve_stats(pgm_server *s, pgm_server_stats *stats);

/* Stop admitting, finish the requests in flight, drop the queue, join the workers. */
void pgm_serve_destroy(pgm_server *s);

/* Thread-local description of the calling thread's last error ("" if none). */
const char *pgm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PGM_H */
