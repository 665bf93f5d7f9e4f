// Range checks of a compiled graph's index arrays (checked mode, PGM_OPT_CHECKED).
//
// Every gather of the LBP kernels (Sec. 4: messages and beliefs addressed through the
// global indices of variable states and factor configurations) reads its addresses from
// these arrays or derives them from the group records. Checked mode verifies every entry
// against the range its consumers assume before the iterations run, so no kernel is
// handed an out-of-range index; a violation is reported, never trapped. The functions
// below are compiled for the host (pgm_audit_desc, CPU tests) and the device (the audit
// kernels), so both sides apply the same rules.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "pgm_internal.h"

namespace pgm {

// Array ids (pgm.h, PGM_FLAG_INDEX): the flat index arrays, then the pools and records.
enum AuditArrayId : int32_t {
    kAuditVsOff = 0,      // vs_off [V+1]: 0..VS
    kAuditVinOff = 1,     // vin_off [V+1]: 0..E
    kAuditVinEs = 2,      // vin_es [E]: 0..ES-1
    kAuditEdgeVs = 3,     // edge_vs [E]: 0..VS-1, with the sign bit set for high-degree variables
    kAuditEdgeVar = 4,    // edge_var [E]: 0..V-1
    kAuditTab4 = 5,       // vin_tab4 [4V]: -1 or 0..ES-1
    kAuditLrPos = 6,      // lr_pos [E]: 0..slots-1
    kAuditParOff = 7,     // paroff_pool: 0..E
    kAuditCfg = 8,        // cfg_pool: state < K of its neighbour (per enumeration group)
    kAuditBs = 9,         // bs_pool: offsets 0..arity n_cfg, configuration ids < n_cfg
    kAuditEnumSeg = 10,   // enumeration group records: every derived range inside its array
    kAuditLogicSeg = 11,  // logical group records
    kAuditVarList = 12,   // variable lists of the variable-pass launches: 0..V-1
    kAuditNumArrays = 13
};

// One flat int32 array and its entries' range [lo, hi). allow_neg: 0 nothing else; 1 -1
// also valid (padding); 2 an entry with the sign bit set also valid when its other bits
// are in range (the marked edges of high-degree variables).
struct AuditArray {
    const int32_t *p;
    int64_t n;
    int64_t lo, hi;
    int32_t allow_neg;
    int32_t id;
};

// Sizes the group records are checked against.
struct AuditSizes {
    int64_t V, VS, E, ES, P;
    int64_t cfg_size, bs_size, paroff_size;
    const uint8_t *cfg_pool;
    const int32_t *bs_pool, *paroff_pool;
};

__host__ __device__ __forceinline__ bool audit_entry_ok(int64_t x, const AuditArray &a) {
    if (x >= a.lo && x < a.hi) return true;
    if (a.allow_neg == 1) return x == -1;
    if (a.allow_neg == 2 && x < 0) {
        const int64_t y = x & 0x7fffffff;
        return y >= a.lo && y < a.hi;
    }
    return false;
}

// A group's lists by output state: es_per_fac + 1 offsets padded to a multiple of four
// entries, then the arity n_cfg list entries, the whole padded to a multiple of four.
__host__ __device__ __forceinline__ int64_t audit_bs_head(const EnumSeg &s) { return (s.es_per_fac + 1 + 3) & ~3; }
__host__ __device__ __forceinline__ int64_t audit_bs_len(const EnumSeg &s) {
    return (audit_bs_head(s) + (int64_t)s.arity * s.n_cfg + 3) & ~(int64_t)3;
}

// An enumeration group record: all its derived index ranges inside their arrays.
__host__ __device__ inline bool audit_enum_seg_ok(const EnumSeg &s, const AuditSizes &z) {
    if (s.n_fac < 0 || s.arity < 1 || s.arity > kMaxArity || s.n_cfg < 1) return false;
    int64_t ksum = 0;
    for (int j = 0; j < s.arity; ++j) {
        if (s.K[j] < 1 || s.K[j] > kMaxStates || s.Koff[j] != ksum) return false;
        ksum += s.K[j];
    }
    if (ksum != s.es_per_fac) return false;
    const int64_t nf = s.n_fac;
    if (s.edge_base < 0 || s.edge_base + nf * s.arity > z.E) return false;
    if (s.es_base < 0 || s.es_base + nf * s.es_per_fac > z.ES) return false;
    if (s.pot_base < 0 || s.pot_base + (s.shared ? (int64_t)s.n_cfg : nf * s.n_cfg) > z.P) return false;
    if (s.cfg_base < 0 || s.cfg_base + (int64_t)s.n_cfg * s.arity > z.cfg_size) return false;
    if (s.bs_base != -1 && (s.bs_base < 0 || s.bs_base + audit_bs_len(s) > z.bs_size)) return false;
    return true;
}

// A logical group record (its last factor's edges inside E and ES).
__host__ __device__ inline bool audit_logic_seg_ok(const LogicSeg &s, const AuditSizes &z) {
    if (s.n_fac < 0 || s.edge_base < 0 || s.es_base < 0 || s.paroff_base < 0) return false;
    if (s.paroff_base + (int64_t)s.n_fac + 1 > z.paroff_size) return false;
    const int64_t np = z.paroff_pool[s.paroff_base + s.n_fac];
    if (np < 0 || s.edge_base + np + s.n_fac > z.E) return false;
    if (s.es_base + 2 * (np + s.n_fac) > z.ES) return false;
    return true;
}

// Entry i of an enumeration group's configuration table: a state of neighbour i % arity.
__host__ __device__ __forceinline__ bool audit_cfg_ok(const EnumSeg &s, int64_t i, const AuditSizes &z) {
    return z.cfg_pool[s.cfg_base + i] < s.K[i % s.arity];
}

// Entry i (0 <= i < audit_bs_len) of a group's lists by output state: an offset into the
// arity n_cfg list entries, padding, or a list entry -- a configuration id, or for packed
// pairwise groups (c << 11) | (Koff[other] + state).
__host__ __device__ __forceinline__ bool audit_bs_ok(const EnumSeg &s, int64_t i, const AuditSizes &z) {
    const int64_t x = z.bs_pool[s.bs_base + i];
    const int64_t n_list = (int64_t)s.arity * s.n_cfg, head = audit_bs_head(s);
    if (i <= s.es_per_fac) return x >= 0 && x <= n_list;
    if (i < head || i >= head + n_list) return true;  // padding, never read
    if (s.packed) return x >= 0 && (x >> 11) < s.n_cfg && (x & 2047) < s.es_per_fac;
    return x >= 0 && x < s.n_cfg;
}

// audit.cu: the audit on the host (first violation in array-id order, -1 if none) and
// on the device (enqueued on s, waits; raises PGM_FLAG_INDEX in *flags on a violation;
// `work` is a device buffer of audit_work_bytes(flat.size()) bytes).
const char *audit_array_name(int id);
void audit_host(const std::vector<AuditArray> &flat, const std::vector<EnumSeg> &esegs,
                const std::vector<LogicSeg> &lsegs, const AuditSizes &z, int32_t *bad_array, int64_t *bad_pos);
size_t audit_work_bytes(size_t n_flat);
cudaError_t audit_device(const std::vector<AuditArray> &flat, const std::vector<std::pair<const void *, int>> &enum_launches,
                         const std::vector<std::pair<const void *, int>> &logic_launches, const AuditSizes &z,
                         uint32_t *flags, char *work, cudaStream_t s, int32_t *bad_array, int64_t *bad_pos);

}  // namespace pgm
