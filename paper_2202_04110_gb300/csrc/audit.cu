// Checked mode (PGM_OPT_CHECKED): the range audit of a graph's index arrays on the
// device before a call's kernels run, and the same audit on the host for a description
// (pgm_audit_desc), both applying the rules of audit.h. A violation is recorded --
// PGM_FLAG_INDEX in the graph's status word, the array, position and value kept for
// pgm_checked_report -- and the call returns PGM_EINVAL before any LBP kernel touches
// the bad index; nothing traps.
#include <algorithm>
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pgm.h"
#include "audit.h"
#include "pgm_internal.h"

namespace pgm {
namespace {

constexpr unsigned long long kNone = ULLONG_MAX;

__global__ void __launch_bounds__(256) k_audit_flat(const AuditArray *__restrict__ arrs,
                                                    unsigned long long *__restrict__ first) {
    const AuditArray a = arrs[blockIdx.y];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        if (!audit_entry_ok(a.p[i], a)) atomicMin(first + a.id, (unsigned long long)i);
}

// One block per enumeration group record: the record, then (if it is sound and the
// group has factors) its configuration table and lists.
__global__ void __launch_bounds__(256) k_audit_enum(const EnumSeg *__restrict__ segs, int64_t seg_pos0, AuditSizes z,
                                                    unsigned long long *__restrict__ first) {
    __shared__ int ok;
    const EnumSeg s = segs[blockIdx.x];
    if (threadIdx.x == 0) {
        ok = audit_enum_seg_ok(s, z) ? 1 : 0;
        if (!ok) atomicMin(first + kAuditEnumSeg, (unsigned long long)(seg_pos0 + blockIdx.x));
    }
    __syncthreads();
    if (!ok || s.n_fac == 0) return;
    const int64_t n_cfg = (int64_t)s.n_cfg * s.arity;
    for (int64_t i = threadIdx.x; i < n_cfg; i += blockDim.x)
        if (!audit_cfg_ok(s, i, z)) atomicMin(first + kAuditCfg, (unsigned long long)(s.cfg_base + i));
    if (s.bs_base < 0) return;
    const int64_t n_bs = audit_bs_len(s);
    for (int64_t i = threadIdx.x; i < n_bs; i += blockDim.x)
        if (!audit_bs_ok(s, i, z)) atomicMin(first + kAuditBs, (unsigned long long)(s.bs_base + i));
}

__global__ void __launch_bounds__(128) k_audit_logic(const LogicSeg *__restrict__ segs, int n_seg, int64_t seg_pos0,
                                                     AuditSizes z, unsigned long long *__restrict__ first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_seg && !audit_logic_seg_ok(segs[i], z))
        atomicMin(first + kAuditLogicSeg, (unsigned long long)(seg_pos0 + i));
}

__global__ void k_audit_flag(uint32_t *flags) { atomicOr(flags, (uint32_t)PGM_FLAG_INDEX); }

const char *const kArrayNames[kAuditNumArrays] = {
    "vs_off", "vin_off", "vin_es", "edge_vs", "edge_var", "vin_tab4", "lr_pos", "paroff_pool",
    "cfg_pool", "bs_pool", "enumeration group records", "logical group records", "variable lists"};

}  // namespace

const char *audit_array_name(int id) { return id >= 0 && id < kAuditNumArrays ? kArrayNames[id] : "?"; }

// Host twin of the device audit: the first violation in array-id order (ids as
// AuditArrayId), -1 if none.
void audit_host(const std::vector<AuditArray> &flat, const std::vector<EnumSeg> &esegs,
                const std::vector<LogicSeg> &lsegs, const AuditSizes &z, int32_t *bad_array, int64_t *bad_pos) {
    std::vector<int64_t> first(kAuditNumArrays, -1);
    auto note = [&](int id, int64_t pos) {
        if (first[id] < 0 || pos < first[id]) first[id] = pos;
    };
    for (const AuditArray &a : flat)
        for (int64_t i = 0; i < a.n; ++i)
            if (!audit_entry_ok(a.p[i], a)) note(a.id, i);
    for (size_t k = 0; k < esegs.size(); ++k) {
        const EnumSeg &s = esegs[k];
        if (!audit_enum_seg_ok(s, z)) {
            note(kAuditEnumSeg, (int64_t)k);
            continue;
        }
        if (s.n_fac == 0) continue;
        for (int64_t i = 0; i < (int64_t)s.n_cfg * s.arity; ++i)
            if (!audit_cfg_ok(s, i, z)) note(kAuditCfg, s.cfg_base + i);
        if (s.bs_base >= 0)
            for (int64_t i = 0; i < audit_bs_len(s); ++i)
                if (!audit_bs_ok(s, i, z)) note(kAuditBs, s.bs_base + i);
    }
    for (size_t k = 0; k < lsegs.size(); ++k)
        if (!audit_logic_seg_ok(lsegs[k], z)) note(kAuditLogicSeg, (int64_t)k);
    *bad_array = -1;
    *bad_pos = -1;
    for (int id = 0; id < kAuditNumArrays; ++id)
        if (first[id] >= 0) {
            *bad_array = id;
            *bad_pos = first[id];
            return;
        }
}

// Device audit: enqueues the checks on s, waits, and returns the first violation in
// array-id order (-1 if none). `work` holds the array list and the result words
// (audit_work_bytes(flat.size())).
size_t audit_work_bytes(size_t n_flat) { return 256 + ((n_flat * sizeof(AuditArray) + 255) / 256) * 256; }

cudaError_t audit_device(const std::vector<AuditArray> &flat, const std::vector<std::pair<const void *, int>> &enum_launches,
                         const std::vector<std::pair<const void *, int>> &logic_launches, const AuditSizes &z,
                         uint32_t *flags, char *work, cudaStream_t s, int32_t *bad_array, int64_t *bad_pos) {
    unsigned long long *first = reinterpret_cast<unsigned long long *>(work);
    AuditArray *arrs = reinterpret_cast<AuditArray *>(work + 256);
    cudaError_t e = cudaMemsetAsync(first, 0xff, kAuditNumArrays * sizeof(unsigned long long), s);
    if (e == cudaSuccess && !flat.empty()) {
        // pageable source: the copy has taken the list when the call returns
        e = cudaMemcpyAsync(arrs, flat.data(), flat.size() * sizeof(AuditArray), cudaMemcpyHostToDevice, s);
        int64_t longest = 1;
        for (const AuditArray &a : flat) longest = std::max(longest, a.n);
        const unsigned bx = (unsigned)std::min<int64_t>((longest + 255) / 256, 4096);
        if (e == cudaSuccess) k_audit_flat<<<dim3(bx, (unsigned)flat.size()), 256, 0, s>>>(arrs, first);
    }
    int64_t pos0 = 0;
    for (const auto &L : enum_launches) {
        if (e != cudaSuccess || L.second <= 0) continue;
        k_audit_enum<<<L.second, 256, 0, s>>>(static_cast<const EnumSeg *>(L.first), pos0, z, first);
        pos0 += L.second;
    }
    pos0 = 0;
    for (const auto &L : logic_launches) {
        if (e != cudaSuccess || L.second <= 0) continue;
        k_audit_logic<<<(L.second + 127) / 128, 128, 0, s>>>(static_cast<const LogicSeg *>(L.first), L.second, pos0, z,
                                                             first);
        pos0 += L.second;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    unsigned long long host[kAuditNumArrays];
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, first, sizeof host, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *bad_array = -1;
    *bad_pos = -1;
    for (int id = 0; id < kAuditNumArrays; ++id)
        if (host[id] != kNone) {
            *bad_array = id;
            *bad_pos = (int64_t)host[id];
            break;
        }
    if (*bad_array >= 0) {
        k_audit_flag<<<1, 1, 0, s>>>(flags);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e;
}

}  // namespace pgm
