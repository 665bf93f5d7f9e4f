// Host graph compiler: validates a pgm_graph_desc and lays the graph out as flat
// int32 index arrays (PGMax, arXiv 2202.04110, Sec. 4: one flat message array, global
// indices of variable states and of the valid factor configurations; no padding).
//
// Outputs (see pgm_internal.h):
//   vs_off[V+1]   first state of each variable (evidence / belief layout)
//   edge_vs[E]    first state of the variable of each edge (factor-major edge order)
//   vin_off/vin_es  CSR from each variable to the first edge-state of each incoming
//                   edge, in ascending edge order (deterministic summation order)
//   cfg_pool      uint8 configuration tables of the enumeration groups
//   bs_pool       the same configurations listed by output edge-state (the gather
//                 order of the block-per-factor form)
//   paroff_pool   par_off arrays of the logical groups
//   per-group segment records with the kernel variant chosen for the group
//   degree buckets of the variables (thread- or block-per-variable)
#include <algorithm>
#include <climits>
#include <cstdio>
#include <limits>
#include <string>

#include "../../include/pgm.h"
#include "pgm_internal.h"

namespace pgm {

namespace {

std::string fmt(const char *f, long long a = 0, long long b = 0, long long c = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, f, a, b, c);
    return buf;
}

constexpr int64_t kI32Max = std::numeric_limits<int32_t>::max();

bool is_dense_pair(const pgm_enum_group &g, int K0, int K1) {
    if (g.arity != 2 || K0 != K1 || g.n_cfg != K0 * K1) return false;
    for (int c = 0; c < g.n_cfg; ++c)
        if (g.cfg[2 * c] != c / K1 || g.cfg[2 * c + 1] != c % K1) return false;
    return true;
}

}  // namespace

std::string compile_graph(const void *const *vdescs, int n_desc, HostLayout *L) {
    if (n_desc < 1) return "no graph descriptions";
    if (!vdescs) return "desc is NULL";
    std::vector<const pgm_graph_desc *> D(n_desc);
    int64_t V = 0;
    for (int m = 0; m < n_desc; ++m) {
        const pgm_graph_desc *d = static_cast<const pgm_graph_desc *>(vdescs[m]);
        if (!d) return fmt("desc %lld is NULL", m);
        if (d->n_vars < 1) return fmt("desc %lld: n_vars must be >= 1", m);
        if (!d->num_states) return fmt("desc %lld: num_states is NULL", m);
        if (d->n_enum_groups < 0 || d->n_logic_groups < 0) return fmt("desc %lld: negative group count", m);
        if (d->n_enum_groups > 0 && !d->enum_groups) return fmt("desc %lld: enum_groups is NULL", m);
        if (d->n_logic_groups > 0 && !d->logic_groups) return fmt("desc %lld: logic_groups is NULL", m);
        D[m] = d;
        V += d->n_vars;
    }
    if (V > kI32Max) return "too many variables for int32 indexing";
    L->V = V;
    L->vs_off.assign(V + 1, 0);
    std::vector<int32_t> Kall(V);
    std::vector<int64_t> voff(n_desc + 1, 0);
    int32_t kmax = 0;
    for (int m = 0; m < n_desc; ++m) {
        voff[m + 1] = voff[m] + D[m]->n_vars;
        for (int64_t v = 0; v < D[m]->n_vars; ++v) {
            int32_t k = D[m]->num_states[v];
            if (k < 1 || k > kMaxStates) return fmt("variable %lld has %lld states (1..256 allowed)", voff[m] + v, k);
            Kall[voff[m] + v] = k;
        }
    }
    for (int64_t v = 0; v < V; ++v) {
        kmax = std::max(kmax, Kall[v]);
        int64_t nx = (int64_t)L->vs_off[v] + Kall[v];
        if (nx > kI32Max) return "too many variable states for int32 indexing";
        L->vs_off[v + 1] = (int32_t)nx;
    }
    L->VS = L->vs_off[V];
    L->max_states = kmax;
    const int32_t *K = Kall.data();

    // ---- count edges and validate groups (variable indices are local to each member)
    int64_t E = 0, F = 0, P = 0, ES = 0;
    for (int m = 0; m < n_desc; ++m) {
        const pgm_graph_desc *d = D[m];
        const int64_t Vm = d->n_vars, vo = voff[m];
        for (int gi = 0; gi < d->n_enum_groups; ++gi) {
            const pgm_enum_group &g = d->enum_groups[gi];
            if (g.arity < 1 || g.arity > kMaxArity) return fmt("enum group %lld: arity %lld not in 1..8", gi, g.arity);
            if (g.n_cfg < 1) return fmt("enum group %lld: n_cfg must be >= 1", gi);
            if (g.n_fac < 0) return fmt("enum group %lld: negative n_fac", gi);
            if (!g.cfg) return fmt("enum group %lld: cfg is NULL", gi);
            if (g.n_fac > 0 && !g.vars) return fmt("enum group %lld: vars is NULL", gi);
            int32_t ksum = 0;
            for (int j = 0; j < g.arity && g.n_fac > 0; ++j) {
                int32_t v0 = g.vars[j];
                if (v0 < 0 || v0 >= Vm) return fmt("enum group %lld: variable %lld out of range", gi, v0);
                ksum += K[vo + v0];
            }
            if (ksum > kEnumBlockStateSum) return fmt("enum group %lld: state sum %lld exceeds 2048", gi, ksum);
            if ((int64_t)g.n_cfg * g.arity > (int64_t)1 << 30)
                return fmt("enum group %lld: n_cfg * arity %lld exceeds 2^30", gi, (int64_t)g.n_cfg * g.arity);
            for (int64_t f = 0; f < g.n_fac; ++f)
                for (int j = 0; j < g.arity; ++j) {
                    int32_t v = g.vars[f * g.arity + j];
                    if (v < 0 || v >= Vm) return fmt("enum group %lld: variable %lld out of range", gi, v);
                    if (K[vo + v] != K[vo + g.vars[j]])
                        return fmt("enum group %lld: factor %lld neighbour %lld differs in state count", gi, f, j);
                }
            for (int c = 0; c < g.n_cfg; ++c)
                for (int j = 0; j < g.arity; ++j) {
                    int32_t s = g.cfg[c * g.arity + j];
                    int32_t kj = g.n_fac > 0 ? K[vo + g.vars[j]] : kMaxStates;
                    if (s < 0 || s >= kj) return fmt("enum group %lld: config %lld state %lld out of range", gi, c, s);
                }
            E += (int64_t)g.n_fac * g.arity;
            ES += (int64_t)g.n_fac * ksum;
            F += g.n_fac;
            P += g.shared_potentials ? g.n_cfg : (int64_t)g.n_cfg * g.n_fac;
        }
        for (int gi = 0; gi < d->n_logic_groups; ++gi) {
            const pgm_logic_group &g = d->logic_groups[gi];
            if (g.kind != PGM_LOGIC_OR && g.kind != PGM_LOGIC_AND && g.kind != PGM_LOGIC_XOR)
                return fmt("logic group %lld: unknown kind %lld", gi, g.kind);
            if (g.n_fac < 0) return fmt("logic group %lld: negative n_fac", gi);
            if (!g.par_off) return fmt("logic group %lld: par_off is NULL", gi);
            if (g.par_off[0] != 0) return fmt("logic group %lld: par_off[0] must be 0", gi);
            for (int64_t f = 0; f < g.n_fac; ++f)
                if (g.par_off[f + 1] < g.par_off[f]) return fmt("logic group %lld: par_off decreases at %lld", gi, f);
            int64_t npar = g.par_off[g.n_fac];
            if (npar > 0 && !g.parents) return fmt("logic group %lld: parents is NULL", gi);
            if (g.n_fac > 0 && !g.child) return fmt("logic group %lld: child is NULL", gi);
            for (int64_t q = 0; q < npar; ++q) {
                int32_t v = g.parents[q];
                if (v < 0 || v >= Vm) return fmt("logic group %lld: parent %lld out of range", gi, v);
                if (K[vo + v] != 2) return fmt("logic group %lld: parent %lld is not binary", gi, v);
            }
            for (int64_t f = 0; f < g.n_fac; ++f) {
                int32_t v = g.child[f];
                if (v < 0 || v >= Vm) return fmt("logic group %lld: child %lld out of range", gi, v);
                if (K[vo + v] != 2) return fmt("logic group %lld: child %lld is not binary", gi, v);
            }
            E += npar + g.n_fac;
            ES += 2 * (npar + g.n_fac);
            F += g.n_fac;
        }
    }
    if (E > kI32Max || ES > kI32Max || P > kI32Max) return "graph too large for int32 indexing";
    L->E = E;
    L->ES = ES;
    L->F = F;
    L->P = P;

    // ---- edges, member by member (each member: enumeration groups, then logical
    // groups), factor-major, with their variable-state offsets
    L->edge_vs.assign(E, 0);
    std::vector<int32_t> edge_es(E + 1, 0), edge_var(E, 0);
    int64_t e = 0, es = 0, pot = 0;
    L->members.clear();
    for (int m = 0; m < n_desc; ++m) {
        const pgm_graph_desc *d = D[m];
        const int32_t vo = (int32_t)voff[m];
        HostMember mem{};
        mem.var_off = vo;
        mem.n_vars = d->n_vars;
        mem.vs_off = L->vs_off[vo];
        mem.n_var_states = L->vs_off[vo + d->n_vars] - L->vs_off[vo];
        mem.edge_off = e;
        mem.es_off = es;
        mem.pot_off = pot;
        for (int gi = 0; gi < d->n_enum_groups; ++gi) {
            const pgm_enum_group &g = d->enum_groups[gi];
            HostEnumGroup hg{};
            EnumSeg &s = hg.seg;
            s.n_fac = g.n_fac;
            s.edge_base = (int32_t)e;
            s.es_base = (int32_t)es;
            s.pot_base = (int32_t)pot;
            s.shared = g.shared_potentials ? 1 : 0;
            s.n_cfg = g.n_cfg;
            s.arity = g.arity;
            L->cfg_pool.resize((L->cfg_pool.size() + 15) & ~(size_t)15, 0);
            if (L->cfg_pool.size() + (size_t)g.n_cfg * g.arity > (size_t)INT32_MAX)
                return "configuration tables exceed 2^31 bytes";
            s.cfg_base = (int32_t)L->cfg_pool.size();
            int32_t off = 0;
            for (int j = 0; j < g.arity; ++j) {
                s.K[j] = g.n_fac > 0 ? K[vo + g.vars[j]] : 1;
                s.Koff[j] = off;
                off += s.K[j];
            }
            s.es_per_fac = off;
            for (int64_t c = 0; c < (int64_t)g.n_cfg * g.arity; ++c) L->cfg_pool.push_back((uint8_t)g.cfg[c]);
            int K0 = s.K[0], K1 = g.arity > 1 ? s.K[1] : 0;
            hg.variant = (off > kMaxStateSum || g.n_cfg > kEnumGenericMaxCfg) ? kEnumBlock : kEnumGeneric;
            if (g.n_fac > 0 && is_dense_pair(g, K0, K1)) {
                // K = 4, 8, 16: thread per factor (the autotuner may switch a launch to
                // another form: K lanes per factor, or for a shared table K / 4 lanes)
                if (K0 == 2) hg.variant = kPair2;
                else if (K0 == 4) hg.variant = kPairT4;
                else if (K0 == 8) hg.variant = kPairT8;
                else if (K0 == 16) hg.variant = kPairT16;
            }
            s.bs_base = -1;
            s.fpb = 1;
            s.lanes = 1;
            s.table_bytes = 0;
            s.packed = 0;
            s.ordered = 0;
            s.member = m;
            s.dense = (g.n_fac > 0 && is_dense_pair(g, K0, K1)) ? 1 : 0;
            if (g.n_fac > 0 && (hg.variant == kEnumGeneric || hg.variant == kEnumBlock)) {
                // configuration lists by output state: for neighbour j and state x, the
                // configurations with state x at j (the block form's gather order)
                // (offsets block padded to a multiple of 4 entries, the whole padded to 4)
                const int64_t nl = (int64_t)g.arity * g.n_cfg, ob = (off + 1 + 3) & ~3;
                const size_t len = (size_t)((ob + nl + 3) & ~(int64_t)3);
                if (L->bs_pool.size() + len > (size_t)INT32_MAX) return "configuration lists exceed 2^31 entries";
                s.bs_base = (int32_t)L->bs_pool.size();
                L->bs_pool.resize(L->bs_pool.size() + len, 0);
                int32_t *bo = L->bs_pool.data() + s.bs_base, *bl = bo + ob;
                for (int j = 0; j < g.arity; ++j)
                    for (int c = 0; c < g.n_cfg; ++c) bo[s.Koff[j] + g.cfg[(int64_t)c * g.arity + j] + 1]++;
                for (int o = 0; o < off; ++o) bo[o + 1] += bo[o];
                std::vector<int32_t> fill(bo, bo + off);
                // pairwise groups with fewer than 2^20 configurations: each entry also
                // carries the other neighbour's state offset (the state sum is <= 2048)
                s.packed = (g.arity == 2 && g.n_cfg < (1 << 20)) ? 1 : 0;
                for (int j = 0; j < g.arity; ++j)
                    for (int c = 0; c < g.n_cfg; ++c) {
                        const int64_t r = (int64_t)c * g.arity;
                        int32_t ent = c;
                        if (s.packed) ent = (c << 11) | (s.Koff[1 - j] + g.cfg[r + 1 - j]);
                        bl[fill[s.Koff[j] + g.cfg[r + j]]++] = ent;
                    }
                // threads per output state from the mean list length (about 8 configs each)
                const int64_t mean = nl / std::max<int32_t>(off, 1);
                while (s.lanes < 32 && mean > 8 * s.lanes) s.lanes *= 2;
                int64_t tb = (((int64_t)g.n_cfg * g.arity + 15) & ~15) + (int64_t)len * 4 +
                             (g.shared_potentials ? (int64_t)g.n_cfg * 4 : 0);
                // packed pairwise lists with a shared table: only the offsets and each list
                // entry beside its configuration's log-potential (one 8-byte read per entry)
                if (g.shared_potentials && s.packed) tb = 4 * ob + 8 * nl;
                s.table_bytes = tb <= kEnumTableSmem ? (int32_t)tb : 0;
            }
            for (int64_t f = 0; f < g.n_fac; ++f)
                for (int j = 0; j < g.arity; ++j) {
                    int32_t v = vo + g.vars[f * g.arity + j];
                    edge_var[e] = v;
                    L->edge_vs[e] = L->vs_off[v];
                    edge_es[e] = (int32_t)es;
                    es += K[v];
                    ++e;
                }
            pot += g.shared_potentials ? g.n_cfg : (int64_t)g.n_cfg * g.n_fac;
            if (g.n_fac > 0) L->enum_groups.push_back(hg);
        }
        for (int gi = 0; gi < d->n_logic_groups; ++gi) {
            const pgm_logic_group &g = d->logic_groups[gi];
            HostLogicGroup hg{};
            LogicSeg &s = hg.seg;
            s.n_fac = g.n_fac;
            s.kind = g.kind;
            s.edge_base = (int32_t)e;
            s.es_base = (int32_t)es;
            s.paroff_base = (int32_t)L->paroff_pool.size();
            s.member = m;
            int32_t mf = 0;
            for (int64_t f = 0; f <= g.n_fac; ++f) L->paroff_pool.push_back(g.par_off[f]);
            for (int64_t f = 0; f < g.n_fac; ++f) {
                mf = std::max(mf, g.par_off[f + 1] - g.par_off[f]);
                for (int32_t q = g.par_off[f]; q < g.par_off[f + 1]; ++q) {
                    int32_t v = vo + g.parents[q];
                    edge_var[e] = v;
                    L->edge_vs[e] = L->vs_off[v];
                    edge_es[e] = (int32_t)es;
                    es += 2;
                    ++e;
                }
                int32_t v = vo + g.child[f];
                edge_var[e] = v;
                L->edge_vs[e] = L->vs_off[v];
                edge_es[e] = (int32_t)es;
                es += 2;
                ++e;
            }
            s.max_fan = mf;
            hg.variant = (mf <= kLogicSmallFan) ? kLogicSmall : kLogicWarp;
            if (g.n_fac > 0) L->logic_groups.push_back(hg);
        }
        mem.n_edges = e - mem.edge_off;
        mem.n_edge_states = es - mem.es_off;
        mem.n_potentials = pot - mem.pot_off;
        L->members.push_back(mem);
    }
    L->cfg_pool.resize((L->cfg_pool.size() + 15) & ~(size_t)15, 0);  // 16-byte copies stay inside

    // ---- variable -> incoming edge-state CSR (ascending edge id)
    L->vin_off.assign(V + 1, 0);
    for (int64_t i = 0; i < E; ++i) L->vin_off[edge_var[i] + 1]++;
    int32_t maxdeg = 0;
    for (int64_t v = 0; v < V; ++v) {
        maxdeg = std::max(maxdeg, L->vin_off[v + 1]);
        L->vin_off[v + 1] += L->vin_off[v];
    }
    L->max_degree = maxdeg;
    L->vin_es.assign(E, 0);
    std::vector<int32_t> fill(L->vin_off.begin(), L->vin_off.end() - 1);
    for (int64_t i = 0; i < E; ++i) L->vin_es[fill[edge_var[i]]++] = edge_es[i];

    // ---- degree buckets; edges of high-degree variables take their variable-to-factor
    // values from their variable's totals (the sign bit of edge_vs marks them)
    if ((int64_t)maxdeg > (int64_t)kVarMaxTiles * kVarTile)
        return fmt("a variable has %lld factors; at most %lld are supported", maxdeg, (long long)kVarMaxTiles * kVarTile);
    for (int kk = 0; kk < kNumVarKinds; ++kk) L->var_bucket[kk].clear();
    for (int64_t v = 0; v < V; ++v) {
        const int32_t k0 = L->vin_off[v], k1 = L->vin_off[v + 1];
        int kind;
        if (k1 - k0 > kVarBlockDegree) {
            kind = kVarBlock;
        } else if (K[v] == 2) {
            bool even = (L->vs_off[v] & 1) == 0;
            for (int32_t k = k0; k < k1 && even; ++k) even = (L->vin_es[k] & 1) == 0;
            kind = even ? kVarBinary : kVarGeneric;
        } else if (K[v] == 4) {
            kind = kVarGroup4;
        } else if (K[v] == 8) {
            kind = kVarGroup8;
        } else if (K[v] == 16) {
            kind = kVarGroup16;
        } else if (K[v] > 16) {
            kind = kVarWarp;
        } else {
            kind = kVarGeneric;
        }
        L->var_bucket[kind].push_back((int32_t)v);
    }
    for (int kk = 0; kk < kNumVarKinds; ++kk) L->var_bucket_identity[kk] = ((int64_t)L->var_bucket[kk].size() == V);
    for (int64_t i = 0; i < E; ++i) {
        int32_t v = edge_var[i];
        // high-degree variables: the sign bit marks the edge (its variable's first state
        // stays in the other bits, where the factor finds the variable's totals)
        if (L->vin_off[v + 1] - L->vin_off[v] > kVarBlockDegree)
            L->edge_vs[i] = (int32_t)((uint32_t)L->vs_off[v] | 0x80000000u);
    }

    // each edge's variable, for the block-per-factor kernel's explicit sums
    L->edge_var.clear();
    bool listed = false;
    for (const HostEnumGroup &hg : L->enum_groups) listed |= hg.seg.bs_base >= 0;
    if (listed) L->edge_var = edge_var;

    L->all_binary = (kmax == 2);
    for (int64_t v = 0; v < V && L->all_binary; ++v)
        if (K[v] != 2) L->all_binary = false;
    // binary graphs whose variables all have at most 4 factors (grids): a padded table of
    // incoming edge-states, one 16-byte row per variable
    L->vin_tab4.clear();
    if (L->all_binary && maxdeg <= 4) {
        L->vin_tab4.assign(4 * V, -1);
        for (int64_t v = 0; v < V; ++v)
            for (int32_t k = L->vin_off[v]; k < L->vin_off[v + 1]; ++k)
                L->vin_tab4[4 * v + (k - L->vin_off[v])] = L->vin_es[k];
    }
    return "";
}

}  // namespace pgm
