// C-ABI entry points (include/pgm.h): graph build and upload, launch planning, the
// flooding LBP run loop, belief read-out and decode.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgm.h"
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

struct pgm_graph {
    int device = 0;
    pgm_info info{};
    DevGraph G{};
    Plan P{};
    void *index_mem = nullptr;    // all index arrays and launch segments
    void *scratch_mem = nullptr;  // ping-pong message buffer, belief buffer, status word
    float *m_tmp = nullptr;
    float *b = nullptr;
    // pgm_infer_host buffers (allocated on first use)
    void *host_io_mem = nullptr;
    float *io_pot = nullptr, *io_ev = nullptr, *io_msgs = nullptr, *io_bel = nullptr;
    int32_t *io_dec = nullptr;
    // per-pass event timing
    int32_t profiling = 0;  // sampling period in iterations, 0 = off
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    int64_t prof_var_launches = 0, prof_factor_launches = 0;
    int32_t var_launches = 0, factor_launches = 0;
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

pgm_status build_plan(const HostLayout &H, pgm_graph *g, Packer &pk, std::vector<size_t> &seg_off,
                      std::vector<int> &seg_kind) {
    // variable pass
    Plan &P = g->P;
    P.kfix = H.all_binary ? 2 : 0;
    {
        VarLaunch L{};
        L.block_mode = 0;
        L.n = (int32_t)H.var_small.size();
        L.threads = 256;
        L.n_blocks = (L.n + 255) / 256;
        L.list = nullptr;
        P.var.push_back(L);
        seg_off.push_back(H.var_small_identity ? (size_t)-1 : pk.add(H.var_small.data(), H.var_small.size()));
        seg_kind.push_back(-1);
    }
    if (!H.var_large.empty()) {
        VarLaunch L{};
        L.block_mode = 1;
        L.n = (int32_t)H.var_large.size();
        L.threads = 256;
        L.n_blocks = L.n;
        P.var.push_back(L);
        seg_off.push_back(pk.add(H.var_large.data(), H.var_large.size()));
        seg_kind.push_back(-2);
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
            P.factor.push_back(L);
            seg_off.push_back(pk.add(segs.data(), segs.size()));
            seg_kind.push_back(variant);
        } else {
            std::vector<EnumSeg> segs;
            int threads = (variant == kPair16 || variant == kEnumGeneric) ? 128 : 256;
            int32_t blk = 0;
            for (const HostEnumGroup &hg : H.enum_groups) {
                if (hg.variant != variant) continue;
                EnumSeg s = hg.seg;
                s.block_begin = blk;
                blk += (s.n_fac + threads - 1) / threads;
                segs.push_back(s);
            }
            if (segs.empty()) continue;
            L.n_seg = (int32_t)segs.size();
            L.n_blocks = blk;
            L.threads = threads;
            P.factor.push_back(L);
            seg_off.push_back(pk.add(segs.data(), segs.size()));
            seg_kind.push_back(variant);
        }
    }
    return PGM_OK;
}

pgm_status take_events(pgm_graph *g, cudaEvent_t *a, cudaEvent_t *b, cudaEvent_t *c) {
    while (g->events.size() < g->events_used + 3) {
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        g->events.push_back(ev);
    }
    *a = g->events[g->events_used];
    *b = g->events[g->events_used + 1];
    *c = g->events[g->events_used + 2];
    g->events_used += 3;
    return PGM_OK;
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

extern "C" {

const char *pgm_last_error(void) { return g_last_error.c_str(); }

pgm_status pgm_build(const pgm_graph_desc *desc, pgm_graph **out) {
    g_last_error.clear();
    if (!out) return fail(PGM_EINVAL, "out is NULL");
    *out = nullptr;
    HostLayout H;
    std::string err = compile_graph(desc, &H);
    if (!err.empty()) return fail(PGM_EINVAL, err);
    pgm_graph *g = new (std::nothrow) pgm_graph();
    if (!g) return fail(PGM_ENOMEM, "host allocation failed");
    cudaError_t ce = cudaGetDevice(&g->device);
    if (ce != cudaSuccess) {
        delete g;
        return cuda_fail(ce, "cudaGetDevice");
    }
    Packer pk;
    size_t o_vs = pk.add(H.vs_off.data(), H.vs_off.size());
    size_t o_vin_off = pk.add(H.vin_off.data(), H.vin_off.size());
    size_t o_vin_es = pk.add(H.vin_es.data(), H.vin_es.size());
    size_t o_edge_vs = pk.add(H.edge_vs.data(), H.edge_vs.size());
    size_t o_cfg = pk.add(H.cfg_pool.data(), H.cfg_pool.size());
    size_t o_po = pk.add(H.paroff_pool.data(), H.paroff_pool.size());
    size_t o_tab4 = H.vin_tab4.empty() ? 0 : pk.add(H.vin_tab4.data(), H.vin_tab4.size());
    std::vector<size_t> seg_off;
    std::vector<int> seg_kind;
    pgm_status st = build_plan(H, g, pk, seg_off, seg_kind);
    if (st != PGM_OK) {
        delete g;
        return st;
    }
    char *dmem = nullptr;
    ce = cudaMalloc(&dmem, pk.host.size());
    if (ce != cudaSuccess) {
        delete g;
        return fail(PGM_ENOMEM, std::string("cudaMalloc(index arrays): ") + cudaGetErrorString(ce));
    }
    ce = cudaMemcpy(dmem, pk.host.data(), pk.host.size(), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        cudaFree(dmem);
        delete g;
        return cuda_fail(ce, "cudaMemcpy(index arrays)");
    }
    g->index_mem = dmem;
    size_t es_bytes = align_up(std::max<int64_t>(H.ES, 1) * sizeof(float), 256);
    size_t vs_bytes = align_up(std::max<int64_t>(H.VS, 1) * sizeof(float), 256);
    size_t hd_bytes = H.var_large.empty() ? 0 : 2 * es_bytes;
    char *smem = nullptr;
    ce = cudaMalloc(&smem, es_bytes + vs_bytes + 256 + hd_bytes);
    if (ce != cudaSuccess) {
        cudaFree(dmem);
        delete g;
        return fail(PGM_ENOMEM, std::string("cudaMalloc(scratch): ") + cudaGetErrorString(ce));
    }
    g->scratch_mem = smem;
    g->m_tmp = reinterpret_cast<float *>(smem);
    g->b = reinterpret_cast<float *>(smem + es_bytes);
    uint32_t *flags = reinterpret_cast<uint32_t *>(smem + es_bytes + vs_bytes);
    ce = cudaMemset(flags, 0, 256);
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
    G.vin_tab4 = H.vin_tab4.empty() ? nullptr : reinterpret_cast<const int4 *>(dmem + o_tab4);
    G.flags = flags;
    G.v2f_hd = hd_bytes ? reinterpret_cast<float *>(smem + es_bytes + vs_bytes + 256) : nullptr;
    // attach device pointers of the launch lists / segments
    size_t vi = 0, fi = 0;
    int max_smem = 0;
    for (size_t k = 0; k < seg_off.size(); ++k) {
        if (seg_kind[k] < 0) {
            VarLaunch &L = g->P.var[vi++];
            L.list = (seg_off[k] == (size_t)-1) ? nullptr : reinterpret_cast<const int32_t *>(dmem + seg_off[k]);
        } else {
            FactorLaunch &L = g->P.factor[fi++];
            L.segs = dmem + seg_off[k];
            max_smem = std::max(max_smem, L.smem);
        }
    }
    ce = prepare_kernels(max_smem);
    if (ce != cudaSuccess) {
        pgm_free(g);
        return cuda_fail(ce, "cudaFuncSetAttribute");
    }
    pgm_info &I = g->info;
    I.n_vars = H.V;
    I.n_var_states = H.VS;
    I.n_factors = H.F;
    I.n_edges = H.E;
    I.n_edge_states = H.ES;
    I.n_potentials = H.P;
    I.max_states = H.max_states;
    I.max_degree = H.max_degree;
    I.device_bytes = (int64_t)(pk.host.size() + es_bytes + vs_bytes + 256 + hd_bytes);
    for (const VarLaunch &L : g->P.var) g->var_launches += (L.n > 0);
    for (const FactorLaunch &L : g->P.factor) g->factor_launches += (L.n_blocks > 0);
    I.launches_per_iter = g->var_launches + g->factor_launches;
    *out = g;
    return PGM_OK;
}

pgm_status pgm_check_desc(const pgm_graph_desc *desc, pgm_info *info) {
    g_last_error.clear();
    if (!info) return fail(PGM_EINVAL, "info is NULL");
    HostLayout H;
    std::string err = compile_graph(desc, &H);
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
    size_t idx = (H.vs_off.size() + H.vin_off.size() + H.vin_es.size() + H.edge_vs.size() +
                  H.paroff_pool.size() + H.var_small.size() + H.var_large.size()) * sizeof(int32_t) +
                 H.cfg_pool.size();
    size_t es_bytes = align_up(std::max<int64_t>(H.ES, 1) * sizeof(float), 256);
    info->device_bytes = (int64_t)(idx + es_bytes + align_up(std::max<int64_t>(H.VS, 1) * sizeof(float), 256) +
                                   256 + (H.var_large.empty() ? 0 : 2 * es_bytes));
    return PGM_OK;
}

void pgm_free(pgm_graph *g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    if (g->index_mem) cudaFree(g->index_mem);
    if (g->scratch_mem) cudaFree(g->scratch_mem);
    if (g->host_io_mem) cudaFree(g->host_io_mem);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    delete g;
}

pgm_status pgm_graph_info(const pgm_graph *g, pgm_info *info) {
    if (!g || !info) return fail(PGM_EINVAL, "NULL argument");
    *info = g->info;
    return PGM_OK;
}

pgm_status pgm_run_bp(pgm_graph *g, const float *log_pot, const float *evidence, float T,
                      float damping, int32_t n_iters, float *msgs, void *stream) {
    pgm_status st = check_run_args(g, log_pot, evidence, T, damping, n_iters, msgs);
    if (st != PGM_OK) return st;
    if (n_iters == 0 || g->info.n_edge_states == 0) return PGM_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return fail(PGM_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *cur = msgs, *nxt = g->m_tmp;
    for (int it = 0; it < n_iters; ++it) {
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
        const bool prof = g->profiling > 0 && (it % g->profiling) == g->profiling - 1;
        if (prof) {
            pgm_status ps = take_events(g, &e0, &e1, &e2);
            if (ps != PGM_OK) return ps;
            cudaEventRecord(e0, s);
        }
        cudaError_t e = launch_var_pass(g->G, g->P, evidence, cur, g->b, kVarIter, nullptr, s);
        if (e != cudaSuccess) return cuda_fail(e, "variable pass launch");
        if (prof) cudaEventRecord(e1, s);
        e = launch_factor_pass(g->G, g->P, log_pot, g->b, evidence, cur, nxt, T, damping, s);
        if (e != cudaSuccess) return cuda_fail(e, "factor pass launch");
        if (prof) {
            cudaEventRecord(e2, s);
            g->prof_var_launches += g->var_launches;
            g->prof_factor_launches += g->factor_launches;
        }
        std::swap(cur, nxt);
    }
    if (cur != msgs) {
        cudaError_t e = cudaMemcpyAsync(msgs, cur, (size_t)g->info.n_edge_states * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(msgs)");
    }
    return PGM_OK;
}

pgm_status pgm_beliefs(pgm_graph *g, const float *evidence, const float *msgs, float *out,
                       int32_t normalise, void *stream) {
    if (!g || !evidence || !out) return fail(PGM_EINVAL, "NULL argument");
    if (!msgs && g->info.n_edge_states > 0) return fail(PGM_EINVAL, "msgs is NULL");
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

pgm_status pgm_pass_times(pgm_graph *g, double *var_ms, double *factor_ms, int64_t *n_var,
                          int64_t *n_factor) {
    if (!g) return fail(PGM_EINVAL, "graph is NULL");
    DeviceGuard dg(g->device);
    double tv = 0.0, tf = 0.0;
    for (size_t k = 0; k + 3 <= g->events_used; k += 3) {
        cudaError_t e = cudaEventSynchronize(g->events[k + 2]);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float a = 0.f, b = 0.f;
        cudaEventElapsedTime(&a, g->events[k], g->events[k + 1]);
        cudaEventElapsedTime(&b, g->events[k + 1], g->events[k + 2]);
        tv += a;
        tf += b;
    }
    if (var_ms) *var_ms = tv;
    if (factor_ms) *factor_ms = tf;
    if (n_var) *n_var = g->prof_var_launches;
    if (n_factor) *n_factor = g->prof_factor_launches;
    g->events_used = 0;
    g->prof_var_launches = g->prof_factor_launches = 0;
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
