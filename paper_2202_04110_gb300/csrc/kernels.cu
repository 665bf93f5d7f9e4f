// CUDA kernels (sm_103a) of one flooding LBP iteration and of the belief read-out.
//
// Method (PGMax, arXiv 2202.04110): log-space loopy belief propagation with parallel
// updates and damping (Sec. 3), enumeration factors over listed configurations
// (Sec. 5.2), logical factors with updates linear in the fan-in (Sec. 3: OR, AND and,
// as the third kind, XOR), flat message arrays updated by gather / scatter (Sec. 4), MAP
// decode (Sec. 5.1).
//
// One iteration is two passes over HBM-resident flat arrays:
//   variable pass  b_v = e_v + sum_{f in N(v)} m_{f->v}            (k_var_*)
//   factor pass    m_{v->f} = b_v - m_{f->v}   (gathered per edge)
//                  mt_{f->i} = factor update (LSE_T over configurations, or the
//                              closed-form logical update)
//                  m_{f->i} <- norm(delta * m_{f->i} + (1 - delta) * norm(mt_{f->i}))
//                  written to the other buffer of a ping-pong pair   (k_pair, k_enum_generic,
//                                                                     k_logic_small, k_logic_warp)
// The path is gather / scatter plus log-sum-exp, bound by HBM bandwidth (or by the SFU
// for large state counts), not a dense contraction: no tensor cores.
//
// Binary pairwise graphs (every variable binary, every factor a 2 x 2 table) run a
// log-ratio form of the same iteration: one float per edge for each message direction,
// the variable pass writing exact leave-one-out variable-to-factor values and the factor
// pass streaming them in factor order (k_var_slot4_lr / k_var_csr_lr, k_pair2_lr).
//
// Numerics: messages and factor arithmetic in FP32. Variable-side sums are compensated
// (float-float) and the beliefs the factor pass reads are stored relative to each
// variable's largest state. An edge whose stored message has an entry that is -inf or
// larger in magnitude than kExactThreshold takes its variable-to-factor values from an
// explicit leave-one-out sum (v2f_slow_edge) instead of b - m -- or, on graphs that keep
// belief residuals (variables of more than 16 states, logical factors) and for finite
// entries, from (b - m) + b_lo, b_lo being what the rounding of b dropped, written by the
// variable pass for every variable that has such an entry; edges of variables with more
// than kVarBlockDegree factors always take the exact value from the variable's per-state
// totals of finite entries and counts of -inf ones (hd_pair).
//
// Launches: the iteration's kernels go out with programmatic dependent launch (each
// waits, pdl_wait, before touching memory), inside CUDA graphs when the graph allows.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>
#include <math_constants.h>

#include "pgm_internal.h"

namespace pgm {
namespace {

constexpr uint32_t kFlagContradiction = 1u;
constexpr uint32_t kFlagNaN = 2u;

#define kNegInf (-CUDART_INF_F)

// Programmatic dependent launch (griddepcontrol): a kernel launched with the
// programmatic-serialization attribute may be scheduled before the previous kernel of
// its stream has finished. pdl_wait() returns once that kernel has completed and its
// writes are visible (at once for a kernel launched without the attribute);
// pdl_launch_dependents() lets the next kernel be scheduled before this one ends.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class Seg>
__device__ __forceinline__ int find_seg(const Seg *__restrict__ segs, int n, int blk) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&segs[mid].block_begin) <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- vector loads / stores with a run-time alignment check -------------------------

template <int N>
__device__ __forceinline__ void load_n(float (&d)[N], const float *__restrict__ p) {
    if constexpr (N % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < N / 4; ++i) {
                float4 q = __ldg(reinterpret_cast<const float4 *>(p) + i);
                d[4 * i] = q.x; d[4 * i + 1] = q.y; d[4 * i + 2] = q.z; d[4 * i + 3] = q.w;
            }
            return;
        }
    }
    if constexpr (N % 2 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 7u) == 0) {
#pragma unroll
            for (int i = 0; i < N / 2; ++i) {
                float2 q = __ldg(reinterpret_cast<const float2 *>(p) + i);
                d[2 * i] = q.x; d[2 * i + 1] = q.y;
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = __ldg(p + i);
}

// Streaming load of data read once per iteration (messages).
template <int N>
__device__ __forceinline__ void load_n_stream(float (&d)[N], const float *__restrict__ p) {
    if constexpr (N % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < N / 4; ++i) {
                float4 q = __ldcs(reinterpret_cast<const float4 *>(p) + i);
                d[4 * i] = q.x; d[4 * i + 1] = q.y; d[4 * i + 2] = q.z; d[4 * i + 3] = q.w;
            }
            return;
        }
    }
    load_n<N>(d, p);
}

template <int N>
__device__ __forceinline__ void store_n(float *__restrict__ p, const float (&s)[N]) {
    if constexpr (N % 4 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
#pragma unroll
            for (int i = 0; i < N / 4; ++i)
                reinterpret_cast<float4 *>(p)[i] = make_float4(s[4 * i], s[4 * i + 1], s[4 * i + 2], s[4 * i + 3]);
            return;
        }
    }
    if constexpr (N % 2 == 0) {
        if ((reinterpret_cast<uintptr_t>(p) & 7u) == 0) {
#pragma unroll
            for (int i = 0; i < N / 2; ++i)
                reinterpret_cast<float2 *>(p)[i] = make_float2(s[2 * i], s[2 * i + 1]);
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = s[i];
}

// ---- compensated (float-float) sums ----------------------------------------------------
// A value hi + lo with |lo| << |hi|: TwoSum keeps the rounding error of every addition,
// giving about 44 significant bits at FP32 speed (FP64 is a small fraction of the FP32
// rate on this GPU). Infinite sums keep lo = 0.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_make(float v) { return FF{v, 0.f}; }

__device__ __forceinline__ FF ff_add(FF a, float v) {
    const float s = a.hi + v;
    if (!isfinite(s)) return FF{s, 0.f};
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (v - bp);
    return FF{s, a.lo + e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    FF r = ff_add(a, b.hi);
    if (!isfinite(r.hi)) return r;
    r.lo += b.lo;
    return r;
}

__device__ __forceinline__ FF ff_shfl_down(FF v, int d) {
    return FF{__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}

// a - b for float-float values, rounded to FP32 (exact up to that rounding when a and b
// are close). -inf - finite = -inf.
__device__ __forceinline__ float ff_diff(FF a, FF b) {
    if (!isfinite(a.hi) || !isfinite(b.hi)) return a.hi - b.hi;
    return (a.hi - b.hi) + (a.lo - b.lo);
}

// a > b, compared exactly on the float-float values
__device__ __forceinline__ bool ff_gt(FF a, FF b) {
    if (a.hi == kNegInf) return false;
    if (b.hi == kNegInf) return true;
    return ff_diff(a, b) > 0.f;
}

// What r = ff_diff(a, b) dropped: (a - b) - r, from the two-sum of the high parts plus
// the low parts; 0 where a or b is not finite.
__device__ __forceinline__ float ff_diff_lo(FF a, FF b, float r) {
    if (!isfinite(a.hi) || !isfinite(b.hi)) return 0.f;
    const float th = a.hi - b.hi, bb = th - a.hi;
    const float te = (a.hi - (th - bb)) + (-b.hi - bb);
    return (th - r) + (te + (a.lo - b.lo));
}

// Belief residuals of a binary variable whose relative beliefs (r0, r1) came from the
// float-float sums (s0, s1): the larger state is exact (0), the other keeps what its
// rounding dropped.
__device__ __forceinline__ void write_b_lo2(float *p, FF s0, FF s1, float r0, float r1) {
    float l0 = 0.f, l1 = 0.f;
    if (r0 != 0.f || r1 != 0.f) {
        if (r1 == 0.f) l0 = ff_diff_lo(s0, s1, r0);
        else l1 = ff_diff_lo(s1, s0, r1);
    }
    reinterpret_cast<float2 *>(p)[0] = make_float2(l0, l1);
}

// ---- variable-to-factor value -------------------------------------------------------

// Explicit leave-one-out values of one edge: v(x) = e_v(x) + sum over the variable's
// other incoming edges of m(x), float-float summed, for all K states of the edge. Used
// when b - m would be unreliable: a stored entry is -inf (-inf - -inf) or very large
// (cancellation). Its per-edge constant differs from the fast path's, which the factor
// update does not see (it is invariant to a constant added to one edge's values).
constexpr float kExactThreshold = 128.f;

__device__ __noinline__ void v2f_slow_edge(const DevGraph G, const float *__restrict__ ev,
                                           const float *__restrict__ m, int vs, int es, int K,
                                           float *__restrict__ out) {
    int lo = 0, hi = G.V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G.vs_off[mid] <= vs) lo = mid;
        else hi = mid - 1;
    }
    const int k0 = G.vin_off[lo], k1 = G.vin_off[lo + 1];
    for (int x = 0; x < K; ++x) {
        FF s = ff_make(ev[vs + x]);
        for (int k = k0; k < k1; ++k) {
            const int e2 = G.vin_es[k];
            if (e2 != es) s = ff_add(s, m[e2 + x]);
        }
        out[x] = s.hi + s.lo;
    }
}

__device__ __forceinline__ bool needs_exact(float mv) { return !(fabsf(mv) <= kExactThreshold); }

// High-degree variables (more than kVarBlockDegree factors; their edges carry edge_vs
// with the sign bit set, the variable's first state in the other bits): the variable pass
// keeps, per state, the float-float sum of the finite evidence and incoming entries and
// the count of the -inf ones (G.hd_b, float4 (hi, lo, count, 0)). An edge's exact
// leave-one-out value is that sum less the edge's own entry -- -inf when another entry
// or the evidence is -inf -- formed in float-float from the four numbers and the entry,
// so that the pass writes nothing per edge. Returned as a (hi, lo) pair.
__device__ __forceinline__ float2 hd_pair(const DevGraph &G, int vs, int x, float mo) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(G.hd_b) + (vs & 0x7fffffff) + x);
    const bool own = (mo == -CUDART_INF_F);
    if (t.z > (own ? 1.f : 0.f)) return make_float2(-CUDART_INF_F, 0.f);
    if (own) return make_float2(t.x, t.y);
    const float sh = t.x - mo;
    if (!isfinite(sh)) return make_float2(sh, 0.f);
    // two-sum of the high parts, then the low part, renormalised
    const float bb = sh - t.x;
    const float err = (t.x - (sh - bb)) + (-mo - bb);
    const float lo = err + t.y;
    const float hi = sh + lo;
    return make_float2(hi, lo - (hi - sh));
}

__device__ __forceinline__ float hd_rel(float2 a, float2 mx) {
    if (!isfinite(a.x) || !isfinite(mx.x)) return a.x - mx.x;
    return (a.x - mx.x) + (a.y - mx.y);
}

__device__ __forceinline__ bool hd_gt(float2 a, float2 b) {
    if (a.x == -CUDART_INF_F) return false;
    if (b.x == -CUDART_INF_F) return true;
    return hd_rel(a, b) > 0.f;
}

// The variable-to-factor values of an edge of a high-degree variable (vs: its edge_vs,
// mo: the edge's stored entries), relative to the edge's largest state.
template <int K>
__device__ __forceinline__ void hd_v2f(const DevGraph &G, int vs, const float (&mo)[K], float (&v)[K]) {
    float2 d[K];
    int arg = 0;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        d[x] = hd_pair(G, vs, x, mo[x]);
        if (x > 0 && hd_gt(d[x], d[arg])) arg = x;
    }
    float2 mx = d[0];
#pragma unroll
    for (int x = 1; x < K; ++x)
        if (x == arg) mx = d[x];
    if (mx.x == -CUDART_INF_F) {
#pragma unroll
        for (int x = 0; x < K; ++x) v[x] = -CUDART_INF_F;
        return;
    }
#pragma unroll
    for (int x = 0; x < K; ++x) v[x] = hd_rel(d[x], mx);
}

// Variable-to-factor values of one K-state edge. Edges of high-degree variables
// (edge_vs < 0) take the exact leave-one-out values from the variable's totals (hd_pair);
// all others use b - m, or the explicit sum when an entry needs it.
template <int K>
__device__ __forceinline__ void gather_v2f(const DevGraph &G, const float *__restrict__ b,
                                           const float *__restrict__ ev, const float *__restrict__ m_old,
                                           int vs, int es, const float (&mo)[K], float (&v)[K]) {
    if (vs < 0) {
        hd_v2f<K>(G, vs, mo, v);
        return;
    }
    bool exact = false;
#pragma unroll
    for (int x = 0; x < K; ++x) exact |= needs_exact(mo[x]);
    if (exact) {
        v2f_slow_edge(G, ev, m_old, vs, es, K, v);
        return;
    }
    load_n<K>(v, b + vs);
#pragma unroll
    for (int x = 0; x < K; ++x) v[x] -= mo[x];
}

// ---- log-sum-exp helpers -------------------------------------------------------------


// T > 0 logical factors: the closed forms chain several exp / log evaluations per edge;
// in FP32 their rounding errors are biased, which long runs on logical-factor graphs
// amplify. They are therefore evaluated in FP64 from the FP32 inputs (the outputs are
// rounded once to FP32). Sums of softplus terms s(x_j / T) are kept as logarithms,
// log A = LSE_j log s(x_j / T), so that very negative log-odds do not underflow.

// log(s(u)), s(u) = log(1 + e^u)
__device__ __forceinline__ double log_softplus_d(double u) {
    if (u < -30.0) return u + log1p(-0.5 * exp(u));
    if (u > 0.0) return log(u + log1p(exp(-u)));
    return log(log1p(exp(u)));
}

__device__ __forceinline__ double lse2_d(double a, double b) {
    const double mx = fmax(a, b);
    if (mx == -CUDART_INF || mx == CUDART_INF) return mx;
    return mx + log1p(exp(fmin(a, b) - mx));
}

// log(e^a - 1) from la = log a
__device__ __forceinline__ double log_expm1_from_log_d(double la) {
    if (la == -CUDART_INF) return -CUDART_INF;
    if (la == CUDART_INF) return CUDART_INF;
    if (la > 0.0) {
        const double a = exp(la);
        return a + log(-expm1(-a));
    }
    if (la > -700.0) {
        const double a = exp(la);
        return la + log(expm1(a) / a);
    }
    return la;
}

// -log(1 - e^{-a}) from la = log a
__device__ __forceinline__ double neg_log_1mexp_from_log_d(double la) {
    if (la == CUDART_INF) return 0.0;
    if (la > 0.0) return -log(-expm1(-exp(la)));
    if (la > -700.0) {
        const double a = exp(la);
        return -la - log(-expm1(-a) / a);
    }
    return -la;
}

// OR update to parent i (T > 0): la = log of the leave-one-out softplus sum (units of
// T), xc = child log-odds.
__device__ __forceinline__ float or_parent_soft(double la, float xc_f, double T) {
    const double xc = xc_f;
    if (la == -CUDART_INF) return xc_f;
    const double y = xc + T * log_expm1_from_log_d(la);
    if (y >= 0.0) return (float)(T * neg_log_1mexp_from_log_d(la) - T * log1p(exp(-y / T)));
    return (float)(xc + T * exp(la) - T * log1p(exp(y / T)));
}

// OR update to parent i (T = 0): S = leave-one-out sum of max(x_j, 0), M = leave-one-out max.
__device__ __forceinline__ float or_parent_max(float S, float M, float xc) {
    float mn = M < 0.f ? M : 0.f;
    float z = xc + S + mn;
    return (z >= 0.f) ? -mn : xc + S;
}

// XOR (parity) factors: the parents and the child have even parity, and a member's
// message depends on all the others alike. With log-odds a_j = x_j / T of the others,
// the product rule of parity checks gives D = prod tanh(-a_j / 2) and the log-odds
// T log((1 - D) / (1 + D)). The magnitude is carried as l_j = log u_j,
// u_j = -log tanh(|a_j| / 2) = log1p(2 / expm1(|a_j|)) (log 2 - |a_j| beyond 30), and the
// others' LSE lambda of the l_j gives log((1 - |D|) / (1 + |D|)) =
// log(-expm1(-e^lambda)) - log1p(e^-e^lambda) (lambda - log 2 once e^lambda < 1e-9); the
// sign is the parity of the others' positive log-odds. T = 0: the others' smallest |x|,
// positive when an odd number of them is positive. FP64 at T > 0, as the OR / AND forms.
__device__ __forceinline__ double xor_log_u(double a) {
    a = fabs(a);
    if (a == 0.0) return CUDART_INF;
    if (isinf(a)) return -CUDART_INF;
    if (a > 30.0) return 0.6931471805599453 - a;
    return log(log1p(2.0 / expm1(a)));
}

// XOR output (T > 0) from the others' LSE lambda and their parity.
__device__ __forceinline__ float xor_out_soft(double lam, bool odd, double T) {
    double r;
    if (lam == CUDART_INF) r = 0.0;
    else if (lam == -CUDART_INF) r = -CUDART_INF;
    else if (lam < -20.7) r = lam - 0.6931471805599453;
    else {
        const double u = exp(lam);
        r = log(-expm1(-u)) - log1p(exp(-u));
    }
    return (float)(T * (odd ? -r : r));
}

__device__ __forceinline__ float xor_out_max(float mn, bool odd) { return odd ? mn : -mn; }

__device__ __forceinline__ float log_odds(float a0, float a1) {
    return (a0 == kNegInf && a1 == kNegInf) ? 0.f : a1 - a0;
}

// ---- message epilogue: normalise, damp, normalise ------------------------------------

template <int K>
__device__ __forceinline__ void normalise_k(float (&t)[K], uint32_t *flags) {
    float mx = kNegInf;
#pragma unroll
    for (int x = 0; x < K; ++x)
        if (t[x] > mx) mx = t[x];
    if (mx == kNegInf) {
#pragma unroll
        for (int x = 0; x < K; ++x) t[x] = 0.f;
        atomicOr(flags, kFlagContradiction);
        return;
    }
#pragma unroll
    for (int x = 0; x < K; ++x) t[x] -= mx;
}

template <int K>
__device__ __forceinline__ void finish_k(float (&t)[K], const float (&mo)[K], float damping,
                                         uint32_t *flags) {
    normalise_k<K>(t, flags);
    if (damping != 0.f) {
        const float w = 1.f - damping;
#pragma unroll
        for (int x = 0; x < K; ++x) t[x] = damping * mo[x] + w * t[x];
    }
    normalise_k<K>(t, flags);
}

__device__ __forceinline__ void normalise_rt(float *t, int K, uint32_t *flags) {
    float mx = kNegInf;
    for (int x = 0; x < K; ++x)
        if (t[x] > mx) mx = t[x];
    if (mx == kNegInf) {
        for (int x = 0; x < K; ++x) t[x] = 0.f;
        atomicOr(flags, kFlagContradiction);
        return;
    }
    for (int x = 0; x < K; ++x) t[x] -= mx;
}

// ---- LSE_T over a row of K values ---------------------------------------------------

template <int K, bool MAXP>
__device__ __forceinline__ float lse_row(const float (&z)[K], float T, float invT) {
    float mx = kNegInf;
#pragma unroll
    for (int y = 0; y < K; ++y) mx = fmaxf(mx, z[y]);
    if (MAXP || mx == kNegInf) return mx;
    if constexpr (K == 2) {
        // log(1 + e^-d), d >= 0, with the SFU exp2 / log2 (absolute error below 3e-7)
        return mx + T * __logf(1.f + __expf((fminf(z[0], z[1]) - mx) * invT));
    } else {
        float s = 0.f;
#pragma unroll
        for (int y = 0; y < K; ++y) s += expf((z[y] - mx) * invT);
        return mx + T * logf(s);
    }
}

// =====================================================================================
// Variable pass
// =====================================================================================

// Multi-sample launches (pgm_run_bp_multi on graphs without the joint log-ratio path;
// the kernels' MS instantiations): gridDim.y samples share the index arrays; a block
// works on sample blockIdx.y, whose
// messages, beliefs, evidence and log-potentials lie at the DevGraph strides (0 for an
// ordinary launch) and whose scratch (exact leave-one-out sums, belief residuals) is the
// sample's slice.
__device__ __forceinline__ int64_t sample_select(DevGraph &G) {
    const int64_t smp = blockIdx.y;
    if (smp != 0) {
        if (G.hd_b) G.hd_b += smp * 4 * G.s_vs;
        if (G.b_lo) G.b_lo += smp * G.s_vs;
    }
    return smp;
}

// Thread per variable (degree <= kVarBlockDegree). Sums are compensated (float-float)
// in ascending edge order. KFIX = 2: every variable binary (states at 2v, edge-states
// even, float2 loads).
template <int KFIX, int MODE, bool MS = false>
__global__ void __launch_bounds__(256) k_var_thread(DevGraph G, const int32_t *__restrict__ list, int n,
                                                    int dense_binary, const float *__restrict__ ev,
                                                    const float *__restrict__ m,
                                                    float *__restrict__ out,
                                                    int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        ev += smp * G.s_vs;
        m += smp * G.s_es;
        out += smp * G.s_vs;
        if (dec) dec += smp * G.V;
    }
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int v = list ? __ldg(list + t) : t;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    if constexpr (KFIX == 2) {
        const int vs = dense_binary ? 2 * v : __ldg(G.vs_off + v);
        const float2 e = __ldg(reinterpret_cast<const float2 *>(ev + vs));
        FF s0 = ff_make(e.x), s1 = ff_make(e.y);
        bool big = false;
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {  // (unrolled: the gathers of later edges issue early)
            const int es = __ldg(G.vin_es + k);
            const float2 q = __ldg(reinterpret_cast<const float2 *>(m + es));
            s0 = ff_add(s0, q.x);
            s1 = ff_add(s1, q.y);
            big |= needs_exact(q.x) | needs_exact(q.y);
        }
        if constexpr (MODE == kVarDecode) {
            dec[v] = ff_gt(s1, s0) ? 1 : 0;
            return;
        }
        if constexpr (MODE == kVarBeliefs) {
            reinterpret_cast<float2 *>(out + vs)[0] = make_float2(s0.hi + s0.lo, s1.hi + s1.lo);
            return;
        }
        // relative to the larger state
        float r0, r1;
        if (s0.hi == kNegInf && s1.hi == kNegInf) {
            r0 = r1 = kNegInf;
        } else if (ff_gt(s1, s0)) {
            r0 = ff_diff(s0, s1);
            r1 = 0.f;
        } else {
            r0 = 0.f;
            r1 = ff_diff(s1, s0);
        }
        if constexpr (MODE == kVarIter) {
            reinterpret_cast<float2 *>(out + vs)[0] = make_float2(r0, r1);
            if (big && G.b_lo != nullptr) write_b_lo2(G.b_lo + vs, s0, s1, r0, r1);
        } else {  // kVarNormalised
            if (r0 == kNegInf && r1 == kNegInf) {
                atomicOr(G.flags, kFlagContradiction);
                reinterpret_cast<float2 *>(out + vs)[0] = make_float2(kNegInf, kNegInf);
            } else {
                if (r0 != r0 || r1 != r1) atomicOr(G.flags, kFlagNaN);
                const float z = log1pf(expf(fminf(r0, r1)));  // the larger state is 0
                reinterpret_cast<float2 *>(out + vs)[0] = make_float2(r0 - z, r1 - z);
            }
        }
    } else {
        const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
        FF best = ff_make(kNegInf);
        int arg = 0;
        bool nan = false, big = false;  // big: an incoming entry needs the exact form
        for (int x = 0; x < K; ++x) {
            FF s = ff_make(__ldg(ev + vs + x));
            for (int k = k0; k < k1; ++k) {
                const float q = __ldg(m + __ldg(G.vin_es + k) + x);
                s = ff_add(s, q);
                big |= needs_exact(q);
            }
            nan |= (s.hi != s.hi);
            if (x == 0 || ff_gt(s, best)) {
                best = s;
                arg = x;
            }
            if constexpr (MODE == kVarBeliefs) out[vs + x] = s.hi + s.lo;
        }
        if constexpr (MODE == kVarDecode) {
            dec[v] = arg;
        } else if constexpr (MODE == kVarIter || MODE == kVarNormalised) {
            // Recompute each state's float-float sum and subtract the best one exactly.
            if (best.hi == kNegInf) {
                if (MODE == kVarNormalised) atomicOr(G.flags, kFlagContradiction);
                for (int x = 0; x < K; ++x) out[vs + x] = kNegInf;
                return;
            }
            if (nan && MODE == kVarNormalised) atomicOr(G.flags, kFlagNaN);
            float acc = 0.f;  // sum over the other states of e^r (the best state adds 1)
            for (int x = 0; x < K; ++x) {
                FF s = ff_make(__ldg(ev + vs + x));
                for (int k = k0; k < k1; ++k) s = ff_add(s, __ldg(m + __ldg(G.vin_es + k) + x));
                const float r = (x == arg) ? 0.f : ff_diff(s, best);
                out[vs + x] = r;
                if (MODE == kVarNormalised && x != arg) acc += expf(r);
                if (MODE == kVarIter && big && G.b_lo != nullptr) G.b_lo[vs + x] = x == arg ? 0.f : ff_diff_lo(s, best, r);
            }
            if constexpr (MODE == kVarNormalised) {
                const float z = log1pf(acc);
                for (int x = 0; x < K; ++x) out[vs + x] -= z;
            }
        }
    }
}

// Warp per variable with more than 16 states (and at most kVarBlockDegree factors): lane
// l takes states l, l + 32, ..; each state's float-float sum adds the evidence and the
// incoming messages in ascending edge order, as k_var_thread does, and the best state is
// the first of the largest, so beliefs, decodes and the iteration's values have the same
// bits (normalised beliefs sum e^r in another order). The iteration also writes b_lo,
// the rounding residual of each value, so that a factor can form b - m without the
// cancellation a large message would cause.
template <int MODE, bool MS = false>
__global__ void __launch_bounds__(256) k_var_warp(DevGraph G, const int32_t *__restrict__ list, int n,
                                                  const float *__restrict__ ev, const float *__restrict__ m,
                                                  float *__restrict__ out, int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        ev += smp * G.s_vs;
        m += smp * G.s_es;
        out += smp * G.s_vs;
        if (dec) dec += smp * G.V;
    }
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= n) return;  // warp-uniform
    const int v = list ? __ldg(list + w) : w;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
    constexpr int R = kMaxStates / 32;
    FF s[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int x = lane + 32 * r;
        s[r] = ff_make(x < K ? __ldg(ev + vs + x) : kNegInf);
    }
    for (int k = k0; k < k1; ++k) {
        const int es = __ldg(G.vin_es + k);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int x = lane + 32 * r;
            if (x < K) s[r] = ff_add(s[r], __ldg(m + es + x));
        }
    }
    FF best = ff_make(kNegInf);
    int arg = K;
    bool nan = false;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int x = lane + 32 * r;
        if (x < K) {
            nan |= (s[r].hi != s[r].hi);
            if (arg == K || ff_gt(s[r], best)) {
                best = s[r];
                arg = x;
            }
        }
    }
    for (int d = 16; d > 0; d >>= 1) {  // first of the largest over the warp
        FF q;
        q.hi = __shfl_xor_sync(0xffffffffu, best.hi, d);
        q.lo = __shfl_xor_sync(0xffffffffu, best.lo, d);
        const int qa = __shfl_xor_sync(0xffffffffu, arg, d);
        if (qa < K && (arg == K || ff_gt(q, best) || (!ff_gt(best, q) && qa < arg))) {
            best = q;
            arg = qa;
        }
    }
    nan = __any_sync(0xffffffffu, nan);
    if constexpr (MODE == kVarDecode) {
        if (lane == 0) dec[v] = arg;
        return;
    }
    if constexpr (MODE == kVarBeliefs) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int x = lane + 32 * r;
            if (x < K) out[vs + x] = s[r].hi + s[r].lo;
        }
        return;
    }
    if (best.hi == kNegInf) {
        if (MODE == kVarNormalised && lane == 0) atomicOr(G.flags, kFlagContradiction);
        for (int x = lane; x < K; x += 32) out[vs + x] = kNegInf;
        return;
    }
    if (nan && MODE == kVarNormalised && lane == 0) atomicOr(G.flags, kFlagNaN);
    float rr[R];
    float acc = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int x = lane + 32 * r;
        rr[r] = (x == arg) ? 0.f : ff_diff(s[r], best);
        if (MODE == kVarNormalised && x < K && x != arg) acc += expf(rr[r]);
        if (MODE == kVarIter && x < K && G.b_lo != nullptr) {
            // s - best as a float-float (two-sum of the high parts plus the low parts),
            // less the rounded value rr: the part of the difference rr dropped
            float lo = 0.f;
            if (x != arg && isfinite(s[r].hi) && isfinite(best.hi)) {
                const float th = s[r].hi - best.hi, bb = th - s[r].hi;
                const float te = (s[r].hi - (th - bb)) + (-best.hi - bb);
                lo = (th - rr[r]) + (te + (s[r].lo - best.lo));
            }
            G.b_lo[vs + x] = lo;
        }
    }
    float z = 0.f;
    if constexpr (MODE == kVarNormalised) {
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        z = log1pf(acc);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int x = lane + 32 * r;
        if (x < K) out[vs + x] = rr[r] - z;
    }
}

// Thread per variable for binary graphs whose variables all have at most 4 factors:
// one 16-byte row of incoming edge-states per variable (-1 = none), all four message
// gathers issued before the compensated sums (in ascending edge order, as the CSR path).
template <int MODE, bool MS = false>
__global__ void __launch_bounds__(256) k_var_tab4(DevGraph G, int n, const float *__restrict__ ev,
                                                  const float *__restrict__ m, float *__restrict__ out,
                                                  int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        ev += smp * G.s_vs;
        m += smp * G.s_es;
        out += smp * G.s_vs;
        if (dec) dec += smp * G.V;
    }
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int4 t = __ldcs(G.vin_tab4 + v);
    const float2 e = __ldcs(reinterpret_cast<const float2 *>(ev) + v);
    const float2 z = make_float2(0.f, 0.f);
    const float2 q0 = t.x >= 0 ? __ldg(reinterpret_cast<const float2 *>(m + t.x)) : z;
    const float2 q1 = t.y >= 0 ? __ldg(reinterpret_cast<const float2 *>(m + t.y)) : z;
    const float2 q2 = t.z >= 0 ? __ldg(reinterpret_cast<const float2 *>(m + t.z)) : z;
    const float2 q3 = t.w >= 0 ? __ldg(reinterpret_cast<const float2 *>(m + t.w)) : z;
    FF s0 = ff_make(e.x), s1 = ff_make(e.y);
    if (t.x >= 0) { s0 = ff_add(s0, q0.x); s1 = ff_add(s1, q0.y); }
    if (t.y >= 0) { s0 = ff_add(s0, q1.x); s1 = ff_add(s1, q1.y); }
    if (t.z >= 0) { s0 = ff_add(s0, q2.x); s1 = ff_add(s1, q2.y); }
    if (t.w >= 0) { s0 = ff_add(s0, q3.x); s1 = ff_add(s1, q3.y); }
    const bool big = needs_exact(q0.x) | needs_exact(q0.y) | needs_exact(q1.x) | needs_exact(q1.y) |
                     needs_exact(q2.x) | needs_exact(q2.y) | needs_exact(q3.x) | needs_exact(q3.y);
    if constexpr (MODE == kVarDecode) {
        dec[v] = ff_gt(s1, s0) ? 1 : 0;
        return;
    }
    if constexpr (MODE == kVarBeliefs) {
        reinterpret_cast<float2 *>(out)[v] = make_float2(s0.hi + s0.lo, s1.hi + s1.lo);
        return;
    }
    float r0, r1;
    if (s0.hi == kNegInf && s1.hi == kNegInf) {
        r0 = r1 = kNegInf;
    } else if (ff_gt(s1, s0)) {
        r0 = ff_diff(s0, s1);
        r1 = 0.f;
    } else {
        r0 = 0.f;
        r1 = ff_diff(s1, s0);
    }
    if constexpr (MODE == kVarIter) {
        reinterpret_cast<float2 *>(out)[v] = make_float2(r0, r1);
        if (big && G.b_lo != nullptr) write_b_lo2(G.b_lo + 2 * v, s0, s1, r0, r1);
    } else {
        if (r0 == kNegInf && r1 == kNegInf) {
            atomicOr(G.flags, kFlagContradiction);
            reinterpret_cast<float2 *>(out)[v] = make_float2(kNegInf, kNegInf);
        } else {
            if (r0 != r0 || r1 != r1) atomicOr(G.flags, kFlagNaN);
            const float zz = log1pf(expf(fminf(r0, r1)));
            reinterpret_cast<float2 *>(out)[v] = make_float2(r0 - zz, r1 - zz);
        }
    }
}

// K/4 lanes per variable (K = 4, 8, 16): lane l owns states 4l .. 4l+3 and sums them
// over the incoming edges (16-byte loads where the offsets allow; a group's lanes read
// 4K contiguous bytes per edge), float-float, ascending edge order; the best state is
// found across the group (the largest rounded sum, lowest state on ties).
template <int K>
__device__ __forceinline__ void group_argmax_vec(float v, int idx, float &mx, int &arg) {
    constexpr int L = K / 4;
    mx = v;
    arg = idx;
#pragma unroll
    for (int d = L / 2; d > 0; d >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, mx, d, L);
        const int oi = __shfl_xor_sync(0xffffffffu, arg, d, L);
        if (ov > mx || (ov == mx && oi < arg)) {
            mx = ov;
            arg = oi;
        }
    }
}

template <int K>
__device__ __forceinline__ float group_sum_vec(float v) {
    constexpr int L = K / 4;
#pragma unroll
    for (int d = L / 2; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d, L);
    return v;
}

template <int K, int MODE, bool MS = false>
__global__ void __launch_bounds__(256) k_var_group(DevGraph G, const int32_t *__restrict__ list, int n,
                                                   const float *__restrict__ ev, const float *__restrict__ m,
                                                   float *__restrict__ out, int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        ev += smp * G.s_vs;
        m += smp * G.s_es;
        out += smp * G.s_vs;
        if (dec) dec += smp * G.V;
    }
    constexpr int L = K / 4;
    const int l = threadIdx.x & (L - 1);
    const int t_raw = (blockIdx.x * blockDim.x + threadIdx.x) / L;
    const bool valid = t_raw < n;
    const int t = valid ? t_raw : n - 1;
    const int v = list ? __ldg(list + t) : t;
    const int vs = __ldg(G.vs_off + v);
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    float e4[4];
    load_n<4>(e4, ev + vs + 4 * l);
    FF s[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) s[j] = ff_make(e4[j]);
    for (int k = k0; k < k1; ++k) {
        float q[4];
        load_n<4>(q, m + __ldg(G.vin_es + k) + 4 * l);
#pragma unroll
        for (int j = 0; j < 4; ++j) s[j] = ff_add(s[j], q[j]);
    }
    // best state: the largest rounded sum, lowest state among equal ones (states whose
    // float-float sums differ by less than one FP32 ulp count as tied)
    float rs[4];
    float lmx = kNegInf;  // NaN states never win; all -inf (or NaN): the lowest state
    int larg = 4 * l;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rs[j] = s[j].hi + s[j].lo;
        if (rs[j] > lmx) {
            lmx = rs[j];
            larg = 4 * l + j;
        }
    }
    float mx;
    int arg;
    group_argmax_vec<K>(lmx, larg, mx, arg);
    if constexpr (MODE == kVarDecode) {
        if (valid && l == 0) dec[v] = arg;
        return;
    }
    if constexpr (MODE == kVarBeliefs) {
        if (valid) store_n<4>(out + vs + 4 * l, rs);
        return;
    }
    // the best state's float-float sum, from the lane that owns it
    const int jb = arg & 3;
    const float bh = jb == 0 ? s[0].hi : jb == 1 ? s[1].hi : jb == 2 ? s[2].hi : s[3].hi;
    const float bl = jb == 0 ? s[0].lo : jb == 1 ? s[1].lo : jb == 2 ? s[2].lo : s[3].lo;
    const FF best{__shfl_sync(0xffffffffu, bh, arg >> 2, L), __shfl_sync(0xffffffffu, bl, arg >> 2, L)};
    const bool dead = best.hi == kNegInf;  // every state -inf
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) r[j] = dead ? kNegInf : (4 * l + j == arg ? 0.f : ff_diff(s[j], best));
    if constexpr (MODE == kVarIter) {
        if (valid) store_n<4>(out + vs + 4 * l, r);
    } else {
        float acc = 0.f;  // sum over the other states of e^r (the best state adds 1)
        bool nan = false;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(4 * l + j == arg || dead)) acc += expf(r[j]);
            nan |= (s[j].hi != s[j].hi);
        }
        acc = group_sum_vec<K>(acc);
        nan = __any_sync(0xffffffffu, nan);
        if (valid && l == 0) {
            if (dead) atomicOr(G.flags, kFlagContradiction);
            if (nan) atomicOr(G.flags, kFlagNaN);
        }
        if (valid) {
            const float z = log1pf(acc);
#pragma unroll
            for (int j = 0; j < 4; ++j) r[j] = dead ? kNegInf : r[j] - z;
            store_n<4>(out + vs + 4 * l, r);
        }
    }
}

// The outputs of a high-degree variable from its float-float totals sb[x] (thread 0):
// the decode, the raw beliefs, or the beliefs relative to the best state (normalised by
// their log-sum-exp in kVarNormalised).
template <int MODE>
__device__ __forceinline__ void var_block_output(const DevGraph &G, const FF *sb, int K, int vs, int v,
                                                 float *__restrict__ out, int32_t *__restrict__ dec) {
    int arg = 0;
    for (int x = 1; x < K; ++x)
        if (ff_gt(sb[x], sb[arg])) arg = x;
    if constexpr (MODE == kVarDecode) {
        dec[v] = arg;
    } else if constexpr (MODE == kVarBeliefs) {
        for (int x = 0; x < K; ++x) out[vs + x] = sb[x].hi + sb[x].lo;
    } else {
        bool nan = false;
        for (int x = 0; x < K; ++x) nan |= (sb[x].hi != sb[x].hi);
        if (MODE == kVarNormalised && nan) atomicOr(G.flags, kFlagNaN);
        if (sb[arg].hi == kNegInf) {
            if (MODE == kVarNormalised) atomicOr(G.flags, kFlagContradiction);
            for (int x = 0; x < K; ++x) out[vs + x] = kNegInf;
            return;
        }
        float acc = 0.f;  // sum over the other states of e^r (the best state adds 1)
        for (int x = 0; x < K; ++x) {
            const float r = (x == arg) ? 0.f : ff_diff(sb[x], sb[arg]);
            out[vs + x] = r;
            if (x != arg) acc += expf(r);
        }
        if (MODE == kVarNormalised) {
            const float z = log1pf(acc);
            for (int x = 0; x < K; ++x) out[vs + x] -= z;
        }
    }
}

// Block-wide float-float sum of v and plain sum of c (a count) in a fixed order; sh holds
// 3 floats per warp.
__device__ __forceinline__ FF block_sum_count(FF v, float &c, float *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        v = ff_add(v, ff_shfl_down(v, d));
        c += __shfl_down_sync(0xffffffffu, c, d);
    }
    if (lane == 0) {
        sh[3 * warp] = v.hi;
        sh[3 * warp + 1] = v.lo;
        sh[3 * warp + 2] = c;
    }
    __syncthreads();
    FF tot = ff_make(0.f);
    c = 0.f;
    for (int w = 0; w < nw; ++w) {
        tot = ff_add(tot, FF{sh[3 * w], sh[3 * w + 1]});
        c += sh[3 * w + 2];
    }
    __syncthreads();
    return tot;
}

// One state's share of a tile of a high-degree variable's incoming edges: kVarItems
// contiguous edges per thread, the finite entries summed in float-float (ascending edge
// order), the -inf ones counted.
__device__ __forceinline__ FF hd_tile_part(const DevGraph &G, const float *__restrict__ m, int k0, int deg,
                                           int tile, int x, float &c) {
    FF s = ff_make(0.f);
    c = 0.f;
    const int base = tile * kVarTile + threadIdx.x * kVarItems;
#pragma unroll
    for (int i = 0; i < kVarItems; ++i) {
        const int k = base + i;
        if (k < deg) {
            const float q = __ldg(m + __ldg(G.vin_es + k0 + k) + x);
            if (q == kNegInf) c += 1.f;
            else s = ff_add(s, q);
        }
    }
    return s;
}

// A state's totals from its evidence and its tile totals (added in tile order): the
// float-float sum of the finite terms and the count of -inf ones; written to G.hd_b in the
// iteration pass. Returns the belief sum: -inf when a term is -inf (NaN stays NaN).
template <int MODE, class TileTot>
__device__ __forceinline__ FF hd_state_total(const DevGraph &G, float e, int n_tiles, TileTot tile, int vs, int x) {
    FF tot = ff_make(e == kNegInf ? 0.f : e);
    float c = e == kNegInf ? 1.f : 0.f;
    for (int t = 0; t < n_tiles; ++t) {
        const float4 q = tile(t);
        tot = ff_add(tot, FF{q.x, q.y});
        c += q.z;
    }
    if (MODE == kVarIter && G.hd_b != nullptr)
        reinterpret_cast<float4 *>(G.hd_b)[vs + x] = make_float4(tot.hi, tot.lo, c, 0.f);
    return (c > 0.f && tot.hi == tot.hi) ? ff_make(kNegInf) : tot;
}

// Block per high-degree variable (more than kVarBlockDegree factors): every state's
// tile totals over tiles of kVarTile edges, then the state's totals (hd_state_total) and
// the outputs of MODE. The split form below computes the same totals in the same order.
template <int MODE, bool MS = false>
__global__ void __launch_bounds__(kVarBlockThreads) k_var_block(DevGraph G, const int32_t *__restrict__ list,
                                                                const float *__restrict__ ev,
                                                                const float *__restrict__ m,
                                                                float *__restrict__ out,
                                                                int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        ev += smp * G.s_vs;
        m += smp * G.s_es;
        out += smp * G.s_vs;
        if (dec) dec += smp * G.V;
    }
    __shared__ float sh[96];
    __shared__ float4 tile_tot[kVarMaxTiles];
    __shared__ FF sb[kMaxStates];
    const int v = list ? __ldg(list + blockIdx.x) : (int)blockIdx.x;
    const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    const int deg = k1 - k0;
    const int n_tiles = (deg + kVarTile - 1) / kVarTile;
    for (int x = 0; x < K; ++x) {
        for (int t = 0; t < n_tiles; ++t) {
            float c;
            const FF s = hd_tile_part(G, m, k0, deg, t, x, c);
            const FF tt = block_sum_count(s, c, sh);
            if (threadIdx.x == 0) tile_tot[t] = make_float4(tt.hi, tt.lo, c, 0.f);
        }
        __syncthreads();
        if (threadIdx.x == 0)
            sb[x] = hd_state_total<MODE>(G, __ldg(ev + vs + x), n_tiles, [&](int t) { return tile_tot[t]; }, vs, x);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    var_block_output<MODE>(G, sb, K, vs, v, out, dec);
}

// The high-degree variables split over tiles of kVarTile edges, a block per tile, for
// more blocks than variables: each block writes its tile's totals of every state to
// G.hd_tot (float4: float-float sum of the finite entries, count of -inf ones), and the
// last of a variable's tiles to finish (a ticket per variable, G.hd_cnt, taken after a
// memory fence and reset by the taker) adds the variable's tile totals in tile order
// (hd_state_total, a thread per state) and writes its outputs -- the same sums in the
// same order as k_var_block. tiles[i] = (position in the variable list, tile, first
// hd_tot entry of the variable, tiles of the variable); a variable's K totals of tile t
// are at hd_tot[first + t K .. + K).
template <int MODE>
__global__ void __launch_bounds__(kVarBlockThreads) k_var_hd(DevGraph G, const int32_t *__restrict__ list,
                                                             const int4 *__restrict__ tiles,
                                                             const float *__restrict__ ev,
                                                             const float *__restrict__ m, float *__restrict__ out,
                                                             int32_t *__restrict__ dec) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    __shared__ float sh[96];
    __shared__ FF sb[kMaxStates];
    __shared__ int s_last;
    const int4 tl = __ldg(tiles + blockIdx.x);
    const int v = list ? __ldg(list + tl.x) : tl.x;
    const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
    const int k0 = __ldg(G.vin_off + v), deg = __ldg(G.vin_off + v + 1) - k0;
    if (K == 2) {  // both states in one pass over the tile (the same sums as hd_tile_part)
        FF s0 = ff_make(0.f), s1 = ff_make(0.f);
        float c0 = 0.f, c1 = 0.f;
        const int base = tl.y * kVarTile + threadIdx.x * kVarItems;
#pragma unroll
        for (int i = 0; i < kVarItems; ++i) {
            const int k = base + i;
            if (k < deg) {
                const int es = __ldg(G.vin_es + k0 + k);
                const float2 q = (es & 1) ? make_float2(__ldg(m + es), __ldg(m + es + 1))
                                          : __ldg(reinterpret_cast<const float2 *>(m + es));
                if (q.x == kNegInf) c0 += 1.f;
                else s0 = ff_add(s0, q.x);
                if (q.y == kNegInf) c1 += 1.f;
                else s1 = ff_add(s1, q.y);
            }
        }
        const FF t0 = block_sum_count(s0, c0, sh);
        const FF t1 = block_sum_count(s1, c1, sh);
        if (threadIdx.x == 0) {
            G.hd_tot[tl.z + tl.y * 2] = make_float4(t0.hi, t0.lo, c0, 0.f);
            G.hd_tot[tl.z + tl.y * 2 + 1] = make_float4(t1.hi, t1.lo, c1, 0.f);
        }
    } else {
        for (int x = 0; x < K; ++x) {
            float c;
            const FF s = hd_tile_part(G, m, k0, deg, tl.y, x, c);
            const FF tt = block_sum_count(s, c, sh);
            if (threadIdx.x == 0) G.hd_tot[tl.z + tl.y * K + x] = make_float4(tt.hi, tt.lo, c, 0.f);
        }
    }
    // the variable's last tile to finish completes it
    if (threadIdx.x == 0) {
        __threadfence();  // this tile's totals are visible before its ticket
        const int ticket = atomicAdd(G.hd_cnt + tl.x, 1);
        s_last = (ticket == tl.w - 1);
        if (s_last) G.hd_cnt[tl.x] = 0;  // for the next launch
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int x = threadIdx.x; x < K; x += blockDim.x)
        sb[x] = hd_state_total<MODE>(G, __ldg(ev + vs + x), tl.w,
                                     [&](int t) { return __ldcg(G.hd_tot + tl.z + t * K + x); }, vs, x);
    __syncthreads();
    if (threadIdx.x != 0) return;
    var_block_output<MODE>(G, sb, K, vs, v, out, dec);
}

// =====================================================================================
// Factor pass: dense pairwise tables (Ising, RBM, Potts), thread per factor
// =====================================================================================

// A batch member whose early exit has frozen it: the factor pass leaves its messages
// alone (a block, or a chunk of the persistent kernel, lies in one member's group).
__device__ __forceinline__ bool member_frozen(const DevGraph &G, int member) {
    return G.frozen != nullptr && __ldg(G.frozen + member) != 0;
}

// A batch run with parameters per member (pgm_run_bp_batch): the member's T, 1 / T and
// damping replace the launch's, and the launch of the other kind (max-product or not)
// skips it. Also true for a frozen member.
template <bool MAXP>
__device__ __forceinline__ bool member_skip(const DevGraph &G, int member, float &T, float &invT, float &damping) {
    if (member_frozen(G, member)) return true;
    if (G.mem_prm != nullptr) {
        const float4 p = __ldg(reinterpret_cast<const float4 *>(G.mem_prm) + member);
        if ((p.x == 0.f) != MAXP) return true;
        T = p.x;
        invT = p.y;
        damping = p.z;
    }
    return false;
}

// The factor-to-variable update of one dense pairwise factor from its two
// variable-to-factor vectors v0, v1 and stored messages mo0, mo1; writes the damped,
// normalised messages.
// Linear-domain form for a table shared by the group (sum-product only): with
// E[x][y] = exp((phi(x,y) - tmax) / T) precomputed per block and w(y) = exp((v(y) - vmax) / T),
//   LSE_T over y of [phi(x,y) + v(y)] = T log(sum_y E[x][y] w(y)) + vmax + tmax.
// The sum is at least E[x][y*] >= exp(-(table range) / T), so nothing underflows when
// the range is at most 60 T (checked per block).
template <int K>
__device__ __forceinline__ void lse_rows_linear(const float *tabE, bool transpose, const float (&v)[K],
                                                float tmax, float T, float invT, float (&o)[K]) {
    float vmax = kNegInf;
#pragma unroll
    for (int y = 0; y < K; ++y) vmax = fmaxf(vmax, v[y]);
    if (vmax == kNegInf) {
#pragma unroll
        for (int x = 0; x < K; ++x) o[x] = kNegInf;
        return;
    }
    float w[K];
#pragma unroll
    for (int y = 0; y < K; ++y) w[y] = __expf((v[y] - vmax) * invT);
#pragma unroll
    for (int x = 0; x < K; ++x) {
        float s = 0.f;
#pragma unroll
        for (int y = 0; y < K; ++y) s = fmaf(transpose ? tabE[y * K + x] : tabE[x * K + y], w[y], s);
        o[x] = T * logf(s) + vmax + tmax;
    }
}

template <int K, bool MAXP>
__device__ __forceinline__ void pair_update(const float *phi_sh, const float *phi_g, float (&v0)[K],
                                            float (&v1)[K], const float (&mo0)[K], const float (&mo1)[K],
                                            float *m_new0, float *m_new1, float T, float invT,
                                            float damping, uint32_t *flags,
                                            const float *tabE = nullptr, float tmax = 0.f) {
    float o0[K], o1[K];
    if (!MAXP && K >= 4 && tabE != nullptr) {
        lse_rows_linear<K>(tabE, false, v1, tmax, T, invT, o0);
        lse_rows_linear<K>(tabE, true, v0, tmax, T, invT, o1);
    } else if constexpr (K <= 4) {
        float phi[K * K];
        if (phi_sh) {
#pragma unroll
            for (int i = 0; i < K * K; ++i) phi[i] = phi_sh[i];
        } else {
            load_n_stream<K * K>(phi, phi_g);
        }
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float z[K];
#pragma unroll
            for (int y = 0; y < K; ++y) z[y] = phi[x * K + y] + v1[y];
            o0[x] = lse_row<K, MAXP>(z, T, invT);
        }
#pragma unroll
        for (int y = 0; y < K; ++y) {
            float z[K];
#pragma unroll
            for (int x = 0; x < K; ++x) z[x] = phi[x * K + y] + v0[x];
            o1[y] = lse_row<K, MAXP>(z, T, invT);
        }
    } else {
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float z[K];
#pragma unroll
            for (int y = 0; y < K; ++y) z[y] = (phi_sh ? phi_sh[x * K + y] : __ldg(phi_g + x * K + y)) + v1[y];
            o0[x] = lse_row<K, MAXP>(z, T, invT);
        }
#pragma unroll
        for (int y = 0; y < K; ++y) {
            float z[K];
#pragma unroll
            for (int x = 0; x < K; ++x) z[x] = (phi_sh ? phi_sh[x * K + y] : __ldg(phi_g + x * K + y)) + v0[x];
            o1[y] = lse_row<K, MAXP>(z, T, invT);
        }
    }
    finish_k<K>(o0, mo0, damping, flags);
    finish_k<K>(o1, mo1, damping, flags);
    store_n<K>(m_new0, o0);
    store_n<K>(m_new1, o1);
}

// Per block: E[i] = exp((tab[i] - tmax) / T) for a shared table, when its range is at
// most 60 T; returns false (E unused) otherwise or for max-product.
template <int K, bool MAXP>
__device__ __forceinline__ bool prepare_linear_table(const float *tab, float *tabE, float *tinfo, float invT) {
    if (MAXP || K < 4) return false;
    if (threadIdx.x == 0) {
        float mx = kNegInf, mn = CUDART_INF_F;
        for (int i = 0; i < K * K; ++i) {
            mx = fmaxf(mx, tab[i]);
            mn = fminf(mn, tab[i]);
        }
        tinfo[0] = mx;
        tinfo[1] = (isfinite(mx) && isfinite(mn) && (mx - mn) * invT <= 60.f) ? 1.f : 0.f;
    }
    __syncthreads();
    const bool use = tinfo[1] != 0.f;
    if (use)
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) tabE[i] = expf((tab[i] - tinfo[0]) * invT);
    __syncthreads();
    return use;
}

// The rare case of a pairwise factor: an edge of a high-degree variable, or a stored
// message entry that is -inf or large. Kept out of line so that the common path holds
// no state across a call.
template <int K, bool MAXP>
__device__ __noinline__ void pair_factor_rare(const DevGraph G, const float *phi_sh, const float *phi_g,
                                              const float *b, const float *ev, const float *m_old,
                                              float *m_new, int vs0, int vs1, int es0, int es1, float T,
                                              float invT, float damping) {
    float mo0[K], mo1[K], v0[K], v1[K];
    load_n<K>(mo0, m_old + es0);
    load_n<K>(mo1, m_old + es1);
    gather_v2f<K>(G, b, ev, m_old, vs0, es0, mo0, v0);
    gather_v2f<K>(G, b, ev, m_old, vs1, es1, mo1, v1);
    pair_update<K, MAXP>(phi_sh, phi_g, v0, v1, mo0, mo1, m_new + es0, m_new + es1, T, invT, damping, G.flags);
}

// Dense pairwise tables (Ising, RBM, Potts): thread per factor.
template <int K, bool MAXP, bool MS = false>
__global__ void __launch_bounds__(K >= 16 ? 128 : 256, K == 2 ? 8 : 1)
k_pair(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
       const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
       float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    __shared__ float tab[K * K];
    __shared__ float tabE[K >= 4 ? K * K : 1];
    __shared__ float tinfo[2];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;  // the whole block
    const int n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared), pot_base = __ldg(&S->pot_base);
    bool linear = false;
    if (shared) {
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) tab[i] = __ldg(pot + pot_base + i);
        __syncthreads();
        linear = prepare_linear_table<K, MAXP>(tab, tabE, tinfo, invT);
    }
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= n_fac) return;
    const int e = __ldg(&S->edge_base) + 2 * f;
    const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
    int vs0, vs1;
    if ((e & 1) == 0) {
        const int2 q = __ldcs(reinterpret_cast<const int2 *>(G.edge_vs + e));
        vs0 = q.x;
        vs1 = q.y;
    } else {
        vs0 = __ldcs(G.edge_vs + e);
        vs1 = __ldcs(G.edge_vs + e + 1);
    }
    const float *phi_sh = shared ? tab : nullptr;
    const float *phi_g = pot + pot_base + (size_t)f * (K * K);
    float mo0[K], mo1[K];
    load_n<K>(mo0, m_old + es0);
    load_n<K>(mo1, m_old + es1);
    // an edge of a high-degree variable is exact from its variable's totals (hd_v2f);
    // only a large or -inf stored entry of another edge takes the out-of-line path
    bool rare = false;
#pragma unroll
    for (int x = 0; x < K; ++x)
        rare |= (vs0 >= 0 && needs_exact(mo0[x])) | (vs1 >= 0 && needs_exact(mo1[x]));
    if (rare) {
        pair_factor_rare<K, MAXP>(G, phi_sh, phi_g, b, ev, m_old, m_new, vs0, vs1, es0, es1, T, invT, damping);
        return;
    }
    float v0[K], v1[K];
    if (vs0 < 0) {
        hd_v2f<K>(G, vs0, mo0, v0);
    } else {
        load_n<K>(v0, b + vs0);
#pragma unroll
        for (int x = 0; x < K; ++x) v0[x] -= mo0[x];
    }
    if (vs1 < 0) {
        hd_v2f<K>(G, vs1, mo1, v1);
    } else {
        load_n<K>(v1, b + vs1);
#pragma unroll
        for (int x = 0; x < K; ++x) v1[x] -= mo1[x];
    }
    pair_update<K, MAXP>(phi_sh, phi_g, v0, v1, mo0, mo1, m_new + es0, m_new + es1, T, invT, damping, G.flags,
                         linear ? tabE : nullptr, linear ? tinfo[0] : 0.f);
}

// ---- K lanes per factor (K = 4, 8, 16): lane x owns state x of both edges ----------

template <int K>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
    for (int d = K / 2; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d, K));
    return v;
}

// normalise-damp-normalise of one edge's state x across its K-lane group
template <int K>
__device__ __forceinline__ float group_finish(float t, float mo, float damping, uint32_t *flags, bool lead) {
    float mx = group_max<K>(t);
    if (mx == kNegInf) {
        t = 0.f;
        if (lead) atomicOr(flags, kFlagContradiction);
    } else {
        t -= mx;
    }
    if (damping != 0.f) t = damping * mo + (1.f - damping) * t;
    mx = group_max<K>(t);
    if (mx == kNegInf) {
        t = 0.f;
        if (lead) atomicOr(flags, kFlagContradiction);
    } else {
        t -= mx;
    }
    return t;
}

// Variable-to-factor value of state x of one edge, for the rare cases: an edge of a
// high-degree variable (float-float leave-one-out pairs, normalised across the group) or
// a stored entry that is -inf or large (explicit leave-one-out sum).
// Called by the K lanes of one group together (gmask = those lanes).
template <int K>
__device__ __noinline__ float group_v2f_rare(const DevGraph G, const float *ev, const float *m_old, int vs,
                                             int es, int x, unsigned gmask) {
    if (vs < 0) {
        const float2 p = hd_pair(G, vs, x, __ldg(m_old + es + x));
        // the edge's largest state, compared exactly on the pairs
        float2 best = p;
#pragma unroll
        for (int d = K / 2; d > 0; d >>= 1) {
            float2 o = make_float2(__shfl_xor_sync(gmask, best.x, d, K), __shfl_xor_sync(gmask, best.y, d, K));
            if (hd_gt(o, best)) best = o;
        }
        if (best.x == -CUDART_INF_F) return -CUDART_INF_F;
        return hd_rel(p, best);
    }
    int lo = 0, hi = G.V - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G.vs_off[mid] <= vs) lo = mid;
        else hi = mid - 1;
    }
    FF s = ff_make(ev[vs + x]);
    for (int k = G.vin_off[lo]; k < G.vin_off[lo + 1]; ++k) {
        const int e2 = G.vin_es[k];
        if (e2 != es) s = ff_add(s, m_old[e2 + x]);
    }
    return s.hi + s.lo;
}

// LSE_T over y of (a(y) + v(y)) where lane y of the group holds v(y); a(y) from `row`.
template <int K, bool MAXP>
__device__ __forceinline__ float group_lse(float v, const float (&a)[K], float T, float invT) {
    float z[K];
    float mx = kNegInf;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        z[y] = a[y] + __shfl_sync(0xffffffffu, v, y, K);
        mx = fmaxf(mx, z[y]);
    }
    if (MAXP || mx == kNegInf) return mx;
    float s = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) s += expf((z[y] - mx) * invT);
    return mx + T * logf(s);
}

// Row stride of the padded exp tables: K + 4 floats keeps rows 16-byte aligned and makes
// the float4 row reads of 8 consecutive lanes fall on distinct bank groups.
template <int K>
constexpr int kRowPad = K + 4;

// Per block, for a shared K x K table phi (row-major, phi[x*K + y]): tab[y*K + x] =
// phi(y, x) (column reads by lane x are contiguous) and tabT[y*K + x] = phi(x, y) (row
// reads by lane x are contiguous); for sum-product, when the table's range is at most
// 60 T (tinfo[1] = 1), E = exp((phi - max phi) / T) padded row-major in tabE (row x of E)
// and tabET (row x of E^T).
template <int K, bool MAXP>
__device__ __forceinline__ void group_tables(const float *__restrict__ phi, float *tab, float *tabT, float *tabE,
                                             float *tabET, float *tinfo, float invT) {
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
        const float p = __ldg(phi + i);
        tab[i] = p;
        tabT[(i % K) * K + i / K] = p;
    }
    if (!MAXP && threadIdx.x < 32) {
        float mx = kNegInf, mn = CUDART_INF_F;
        for (int i = threadIdx.x; i < K * K; i += 32) {
            const float p = __ldg(phi + i);
            mx = fmaxf(mx, p);
            mn = fminf(mn, p);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, d));
        }
        if (threadIdx.x == 0) {
            tinfo[0] = mx;
            tinfo[1] = (isfinite(mx) && isfinite(mn) && (mx - mn) * invT <= 60.f) ? 1.f : 0.f;
        }
    }
    __syncthreads();
    if (!MAXP && tinfo[1] != 0.f) {
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
            const int r = i / K, c = i % K;
            const float e = expf((tab[i] - tinfo[0]) * invT);
            tabE[r * kRowPad<K> + c] = e;   // E(r, c)
            tabET[c * kRowPad<K> + r] = e;  // E^T(c, r)
        }
    }
    __syncthreads();
}

// Dense pairwise tables with K states (Potts): K lanes per factor. The launch's
// factors are cut into chunks of blockDim / K factors ("virtual blocks", numbered as in
// the segments' block ranges); each physical block walks a contiguous range of chunks
// and rebuilds its shared-memory tables only when the chunk's group changes, so the
// per-table work is paid once per block rather than once per chunk.
template <int K, bool MAXP, bool MS = false>
__global__ void __launch_bounds__(256, 4)
k_pair_group(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, int n_vblocks, const float *__restrict__ pot,
             const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
             float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    __shared__ float tab[K * K], tabT[K * K];
    __shared__ __align__(16) float tabE[MAXP ? 4 : K * kRowPad<K>];
    __shared__ __align__(16) float tabET[MAXP ? 4 : K * kRowPad<K>];
    __shared__ __align__(16) float wsh[MAXP ? 4 : 2 * 256];  // per lane: w1, then w0 at +blockDim
    __shared__ float tinfo[2];
    const int per = (n_vblocks + gridDim.x - 1) / gridDim.x;
    const int vb_begin = blockIdx.x * per;
    const int vb_end = min(vb_begin + per, n_vblocks);
    const int x = threadIdx.x & (K - 1);
    int cur = -1;
    int si = vb_begin < vb_end ? find_seg(segs, n_seg, vb_begin) : 0;
    bool linear = false, shared = false;
    // chunk coordinates and the loads that do not depend on other loads, one chunk ahead
    int nsi = si, nvs0 = 0, nvs1 = 0;
    float nmo0 = 0.f, nmo1 = 0.f;
    auto fetch = [&](int vb, int &s_idx, int &vs0_, int &vs1_, float &mo0_, float &mo1_) {
        while (s_idx + 1 < n_seg && __ldg(&segs[s_idx + 1].block_begin) <= vb) ++s_idx;
        const EnumSeg *Sx = segs + s_idx;
        const int nf = __ldg(&Sx->n_fac);
        int ff = (vb - __ldg(&Sx->block_begin)) * (blockDim.x / K) + threadIdx.x / K;
        if (ff >= nf) ff = nf - 1;
        const int ee = __ldg(&Sx->edge_base) + 2 * ff;
        const int e0 = __ldg(&Sx->es_base) + 2 * K * ff;
        vs0_ = __ldg(G.edge_vs + ee);
        vs1_ = __ldg(G.edge_vs + ee + 1);
        mo0_ = __ldg(m_old + e0 + x);
        mo1_ = __ldg(m_old + e0 + K + x);
    };
    if (vb_begin < vb_end) fetch(vb_begin, nsi, nvs0, nvs1, nmo0, nmo1);
    for (int vb = vb_begin; vb < vb_end; ++vb) {
        si = nsi;
        const int vs0 = nvs0, vs1 = nvs1;
        const float mo0 = nmo0, mo1 = nmo1;
        const EnumSeg *S = segs + si;
        const int n_fac = __ldg(&S->n_fac), pot_base = __ldg(&S->pot_base);
        // beliefs of this chunk, then the next chunk's independent loads
        const bool fast0 = vs0 >= 0, fast1 = vs1 >= 0;
        const float bb0 = fast0 ? __ldg(b + vs0 + x) : 0.f;
        const float bb1 = fast1 ? __ldg(b + vs1 + x) : 0.f;
        if (vb + 1 < vb_end) fetch(vb + 1, nsi, nvs0, nvs1, nmo0, nmo1);
        if (member_skip<MAXP>(G, S->member, T, invT, damping)) continue;  // uniform across the block
        if (si != cur) {  // uniform across the block
            cur = si;
            shared = __ldg(&S->shared) != 0;
            __syncthreads();
            if (shared) {
                group_tables<K, MAXP>(pot + pot_base, tab, tabT, tabE, tabET, tinfo, invT);
                linear = !MAXP && tinfo[1] != 0.f;
            } else {
                linear = false;
            }
        }
        const int f_raw = (vb - __ldg(&S->block_begin)) * (blockDim.x / K) + threadIdx.x / K;
        const bool valid = f_raw < n_fac;
        const int f = valid ? f_raw : n_fac - 1;  // idle lanes shadow the last factor, store nothing
        const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
        // rare-case vote within the group (uniform across its K lanes): any state of the
        // edge needing the exact path
        const unsigned gmask = ((1u << K) - 1u) << ((threadIdx.x & 31) & ~(K - 1));
        const unsigned b0 = __ballot_sync(0xffffffffu, needs_exact(mo0)) & gmask;
        const unsigned b1 = __ballot_sync(0xffffffffu, needs_exact(mo1)) & gmask;
        float v0, v1;
        if (vs0 < 0 || b0) v0 = group_v2f_rare<K>(G, ev, m_old, vs0, es0, x, gmask);
        else v0 = bb0 - mo0;
        if (vs1 < 0 || b1) v1 = group_v2f_rare<K>(G, ev, m_old, vs1, es1, x, gmask);
        else v1 = bb1 - mo1;
        float o0, o1;
        if (!MAXP && linear) {
            // to variable 0, state x: row x of E against w1; to variable 1: column x against w0
            const float vmax1 = group_max<K>(v1), vmax0 = group_max<K>(v0);
            const float w1 = vmax1 == kNegInf ? 0.f : __expf((v1 - vmax1) * invT);
            const float w0 = vmax0 == kNegInf ? 0.f : __expf((v0 - vmax0) * invT);
            // stage the group's weights; the group's lanes are in one warp
            const int gbase = threadIdx.x & ~(K - 1);
            wsh[threadIdx.x] = w1;
            wsh[blockDim.x + threadIdx.x] = w0;
            __syncwarp();
            const float4 *er = reinterpret_cast<const float4 *>(tabE + x * kRowPad<K>);   // row x of E
            const float4 *ec = reinterpret_cast<const float4 *>(tabET + x * kRowPad<K>);  // row x of E^T
            const float4 *w1v = reinterpret_cast<const float4 *>(wsh + gbase);
            const float4 *w0v = reinterpret_cast<const float4 *>(wsh + blockDim.x + gbase);
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const float4 a = er[j], wa = w1v[j], c = ec[j], wc = w0v[j];
                s0 = fmaf(a.x, wa.x, fmaf(a.y, wa.y, fmaf(a.z, wa.z, fmaf(a.w, wa.w, s0))));
                s1 = fmaf(c.x, wc.x, fmaf(c.y, wc.y, fmaf(c.z, wc.z, fmaf(c.w, wc.w, s1))));
            }
            __syncwarp();
            o0 = vmax1 == kNegInf ? kNegInf : T * logf(s0) + vmax1 + tinfo[0];
            o1 = vmax0 == kNegInf ? kNegInf : T * logf(s1) + vmax0 + tinfo[0];
        } else {
            float row[K], col[K];
            const float *phi_g = pot + pot_base + (size_t)f * (K * K);
#pragma unroll
            for (int y = 0; y < K; ++y) {
                row[y] = shared ? tabT[y * K + x] : __ldg(phi_g + x * K + y);
                col[y] = shared ? tab[y * K + x] : __ldg(phi_g + y * K + x);
            }
            o0 = group_lse<K, MAXP>(v1, row, T, invT);
            o1 = group_lse<K, MAXP>(v0, col, T, invT);
        }
        const bool lead = valid && x == 0;
        o0 = group_finish<K>(o0, mo0, damping, G.flags, lead);
        o1 = group_finish<K>(o1, mo1, damping, G.flags, lead);
        if (valid) {
            m_new[es0 + x] = o0;
            m_new[es1 + x] = o1;
        }
    }
}

// ---- K-state pairwise tables, thread per factor ------------------------------------

// One direction of a K-state pairwise factor, thread-local: o(x) = LSE_T (or max) over y
// of phi(x, y) + v(y) for the message to variable 0 (TR = false, rows of phi), or of
// phi(y, x) + v(y) for the message to variable 1 (TR = true, columns). Linear form for a
// shared table with E = exp((phi - tmax) / T) (tabE row-major E, tabET row-major E^T):
// o(x) = T log(sum_y E(x, y) w(y)) + vmax + tmax with w(y) = exp((v(y) - vmax) / T), the
// rows read as float4 (every thread of the block reads the same row: a broadcast).
template <int K, bool MAXP, bool TR>
__device__ __forceinline__ void pair_dir_thr(float (&v)[K], float (&o)[K], bool linear, const float *tabE,
                                             const float *phi, bool phi_shared, float tmax, float T,
                                             float invT) {
    if (!MAXP && linear) {
        float vmax = kNegInf;
#pragma unroll
        for (int y = 0; y < K; ++y) vmax = fmaxf(vmax, v[y]);
        if (vmax == kNegInf) {
#pragma unroll
            for (int x = 0; x < K; ++x) o[x] = kNegInf;
            return;
        }
#pragma unroll
        for (int y = 0; y < K; ++y) v[y] = __expf((v[y] - vmax) * invT);  // w(y), in (0, 1]
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const float4 *row = reinterpret_cast<const float4 *>(tabE + x * K);
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const float4 a = row[j];
                s = fmaf(a.x, v[4 * j], fmaf(a.y, v[4 * j + 1], fmaf(a.z, v[4 * j + 2], fmaf(a.w, v[4 * j + 3], s))));
            }
            o[x] = T * logf(s) + vmax + tmax;
        }
    } else {
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float z[K];
#pragma unroll
            for (int y = 0; y < K; ++y) {
                const int i = TR ? y * K + x : x * K + y;
                z[y] = (phi_shared ? phi[i] : __ldg(phi + i)) + v[y];
            }
            o[x] = lse_row<K, MAXP>(z, T, invT);
        }
    }
}

// Dense K-state pairwise tables (Potts, K = 4, 8, 16), thread per factor: the thread
// keeps the factor's two stored messages and one variable-to-factor vector in registers
// and forms the K x K table product itself, one direction at a time (no cross-lane
// traffic, so the per-factor work is the product's K^2 multiply-adds plus 2K
// exponentials and logarithms per direction). Shared tables are staged per block in
// shared memory (with E and E^T for the linear form); per-factor tables are read from
// the factor's own K*K entries. The rare cases (an edge of a high-degree variable, a
// stored entry that is -inf or large) go to pair_factor_rare.
template <int K, bool MAXP, bool MS = false>
__global__ void __launch_bounds__(K >= 16 ? 128 : 256)
k_pair_thr(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
           const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
           float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    __shared__ float tab[K * K];
    __shared__ __align__(16) float tabE[MAXP ? 4 : K * K];
    __shared__ __align__(16) float tabET[MAXP ? 4 : K * K];
    __shared__ float tinfo[2];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;  // the whole block
    const int n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared), pot_base = __ldg(&S->pot_base);
    bool linear = false;
    if (shared) {  // uniform over the block (a block lies in one segment)
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) tab[i] = __ldg(pot + pot_base + i);
        __syncthreads();
        linear = prepare_linear_table<K, MAXP>(tab, tabE, tinfo, invT);
        if (linear) {
            for (int i = threadIdx.x; i < K * K; i += blockDim.x) tabET[(i % K) * K + i / K] = tabE[i];
            __syncthreads();
        }
    }
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= n_fac) return;
    const int e = __ldg(&S->edge_base) + 2 * f;
    const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
    const int vs0 = __ldg(G.edge_vs + e), vs1 = __ldg(G.edge_vs + e + 1);
    const float *phi = shared ? tab : pot + pot_base + (size_t)f * (K * K);
    const float tmax = linear ? tinfo[0] : 0.f;
    float mo0[K], mo1[K];
    load_n_stream<K>(mo0, m_old + es0);
    load_n_stream<K>(mo1, m_old + es1);
    bool rare = (vs0 < 0) | (vs1 < 0);
#pragma unroll
    for (int x = 0; x < K; ++x) rare |= needs_exact(mo0[x]) | needs_exact(mo1[x]);
    if (rare) {
        pair_factor_rare<K, MAXP>(G, shared ? tab : nullptr, pot + pot_base + (size_t)f * (K * K), b, ev, m_old,
                                  m_new, vs0, vs1, es0, es1, T, invT, damping);
        return;
    }
    float v[K], o[K];
    // to variable 0: rows of phi against v1 = b1 - m1
    load_n<K>(v, b + vs1);
#pragma unroll
    for (int y = 0; y < K; ++y) v[y] -= mo1[y];
    pair_dir_thr<K, MAXP, false>(v, o, linear, tabE, phi, shared, tmax, T, invT);
    finish_k<K>(o, mo0, damping, G.flags);
    store_n<K>(m_new + es0, o);
    // to variable 1: columns of phi against v0 = b0 - m0
    load_n<K>(v, b + vs0);
#pragma unroll
    for (int y = 0; y < K; ++y) v[y] -= mo0[y];
    pair_dir_thr<K, MAXP, true>(v, o, linear, tabET, phi, shared, tmax, T, invT);
    finish_k<K>(o, mo1, damping, G.flags);
    store_n<K>(m_new + es1, o);
}

// ---- K-state pairwise tables, a thread per factor and direction ------------------------
//
// The two directions of a pairwise factor are independent given the stored messages: the
// message to variable 0 needs only v1 = b1 - m1 and the old m0 (for damping), the message
// to variable 1 only v0 and m1. Here a pair of warps takes 32 factors, the even warp the
// direction to variable 0 and the odd one the direction to variable 1, so a thread holds
// one input vector, one output and one old message (3K values instead of the thread
// form's 4K plus a second output) and twice as many factors are in flight per SM at the
// same arithmetic per factor. Each thread runs the thread form's direction code on the
// same inputs, so both forms give the same bits; a factor with a rare case (an edge of a
// high-degree variable, a stored entry that is -inf or large) is finished whole by the
// even warp's thread through pair_factor_rare, as in the thread form.
template <int K, bool MAXP, bool MS = false>
__global__ void __launch_bounds__(256, K >= 16 ? 3 : 5)
k_pair_dir(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
           const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
           float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    __shared__ float tab[K * K];
    __shared__ __align__(16) float tabE[MAXP ? 4 : K * K];
    __shared__ __align__(16) float tabET[MAXP ? 4 : K * K];
    __shared__ float tinfo[2];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;  // the whole block
    const int n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared), pot_base = __ldg(&S->pot_base);
    bool linear = false;
    if (shared) {  // uniform over the block (a block lies in one segment)
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) tab[i] = __ldg(pot + pot_base + i);
        __syncthreads();
        linear = prepare_linear_table<K, MAXP>(tab, tabE, tinfo, invT);
        if (linear) {
            for (int i = threadIdx.x; i < K * K; i += blockDim.x) tabET[(i % K) * K + i / K] = tabE[i];
            __syncthreads();
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = warp & 1;  // d: warp-uniform
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * (blockDim.x >> 1) + (warp >> 1) * 32 + lane;
    if (f >= n_fac) return;
    const int e = __ldg(&S->edge_base) + 2 * f;
    const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
    const int vs0 = __ldg(G.edge_vs + e), vs1 = __ldg(G.edge_vs + e + 1);
    const float *phi = shared ? tab : pot + pot_base + (size_t)f * (K * K);
    // this thread's output edge (target) and input edge (source)
    const int es_t = d ? es1 : es0, es_s = d ? es0 : es1, vs_s = d ? vs0 : vs1;
    float mo_t[K], v[K];
    load_n<K>(mo_t, m_old + es_t);
    load_n<K>(v, m_old + es_s);
    bool rare = (vs0 < 0) | (vs1 < 0);
#pragma unroll
    for (int x = 0; x < K; ++x) rare |= needs_exact(mo_t[x]) | needs_exact(v[x]);
    if (rare) {  // both warps see the same rare flag; the even one finishes the factor
        if (d == 0)
            pair_factor_rare<K, MAXP>(G, shared ? tab : nullptr, pot + pot_base + (size_t)f * (K * K), b, ev, m_old,
                                      m_new, vs0, vs1, es0, es1, T, invT, damping);
        return;
    }
    const float tmax = linear ? tinfo[0] : 0.f;
    float bs[K], o[K];
    load_n<K>(bs, b + vs_s);
#pragma unroll
    for (int y = 0; y < K; ++y) v[y] = bs[y] - v[y];
    if (d == 0)  // to variable 0: rows of phi against v1
        pair_dir_thr<K, MAXP, false>(v, o, linear, tabE, phi, shared, tmax, T, invT);
    else  // to variable 1: columns of phi against v0
        pair_dir_thr<K, MAXP, true>(v, o, linear, tabET, phi, shared, tmax, T, invT);
    finish_k<K>(o, mo_t, damping, G.flags);
    store_n<K>(m_new + es_t, o);
}

// ---- K / 4 lanes per factor, four consecutive states each (K = 8, 16, shared tables) ----
//
// The factor's L = K / 4 lanes form an aligned group of a warp: lane q loads the states
// 4q..4q+3 of both stored messages and both beliefs (16-byte loads; the group reads each
// vector as one contiguous run) and computes the outputs of those four states in both
// directions. The input vector of a direction is exchanged through the group's slot of
// shared memory, and each output state's row of the table (rows swizzled in 16-byte
// chunks, conflict-free float4 reads) is dotted with it. Per factor this spreads the thread form's work over L
// lanes with a quarter of its registers, so four times as many factors are in flight per
// SM. The arithmetic is the thread form's, term for term and in the same order (the
// table rows in the same float4 chunks, the maxima exact), so both forms give the same
// bits. The rare cases (an edge of a high-degree variable, a stored entry that is -inf
// or large) go to pair_factor_rare on the group's first lane.

// Shared tables of the K / 4-lane form: row x of a K x K table holds its 16-byte chunk j
// at chunk slot j ^ ((x >> 2) & (K / 4 - 1)), so that the group's lanes, reading rows
// 4q + i (q = 0 .. K/4 - 1) at the same time, hit distinct bank groups.
template <int K>
__device__ __forceinline__ int qtab_index(int x, int y) {
    return x * K + 4 * ((y >> 2) ^ ((x >> 2) & (K / 4 - 1))) + (y & 3);
}

// Four consecutive floats of global memory: one 16-byte access when the address is
// 16-byte aligned (a batch member's arrays start wherever the previous member's end),
// else four 4-byte accesses. Written as PTX so that each branch issues exactly these
// accesses (the compiler may not merge the 4-byte ones into wider ones).
__device__ __forceinline__ float4 ld4(const float *p, bool stream) {
    float4 v;
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        if (stream)
            asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        else
            asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
        return v;
    }
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v.x) : "l"(p));
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v.y) : "l"(p + 1));
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v.z) : "l"(p + 2));
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v.w) : "l"(p + 3));
    return v;
}

__device__ __forceinline__ void st4(float *p, float4 v) {
    if ((reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                     : "memory");
        return;
    }
    asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v.x) : "memory");
    asm volatile("st.global.f32 [%0], %1;" ::"l"(p + 1), "f"(v.y) : "memory");
    asm volatile("st.global.f32 [%0], %1;" ::"l"(p + 2), "f"(v.z) : "memory");
    asm volatile("st.global.f32 [%0], %1;" ::"l"(p + 3), "f"(v.w) : "memory");
}

template <int L>
__device__ __forceinline__ float quad_max(float v) {
#pragma unroll
    for (int d = L / 2; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d, L));
    return v;
}

// normalise the group's K values (four per lane) by their maximum; all -inf becomes 0
template <int L>
__device__ __forceinline__ void quad_normalise(float4 &t, uint32_t *flags, bool lead) {
    const float mx = quad_max<L>(fmaxf(fmaxf(t.x, t.y), fmaxf(t.z, t.w)));
    if (mx == kNegInf) {
        t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lead) atomicOr(flags, kFlagContradiction);
        return;
    }
    t.x -= mx;
    t.y -= mx;
    t.z -= mx;
    t.w -= mx;
}

// One direction: the outputs of states 4q..4q+3 from the input vector v (this lane's
// four states) against the rows of `rows` (a padded K x K table: E or E^T for the linear
// form, phi or phi^T otherwise). xs is the group's exchange slot (K floats).
template <int K, bool MAXP>
__device__ __forceinline__ float4 quad_dir(float4 v, bool linear, const float *rows, float *xs, int q, float tmax,
                                          float T, float invT) {
    constexpr int L = K / 4;
    float4 o;
    if (!MAXP && linear) {
        const float vm = quad_max<L>(fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
        // all -inf: w = 0 and every output -inf, as in the thread form
        const float vmax = vm;
        float4 w;
        if (vmax == kNegInf) {
            w = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            w = make_float4(__expf((v.x - vmax) * invT), __expf((v.y - vmax) * invT), __expf((v.z - vmax) * invT),
                            __expf((v.w - vmax) * invT));
        }
        reinterpret_cast<float4 *>(xs)[q] = w;
        __syncwarp();
        float wa[K];
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            const float4 a = reinterpret_cast<const float4 *>(xs)[j];
            wa[4 * j] = a.x; wa[4 * j + 1] = a.y; wa[4 * j + 2] = a.z; wa[4 * j + 3] = a.w;
        }
        __syncwarp();
        float out[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = 4 * q + i, sw = (x >> 2) & (K / 4 - 1);
            const float4 *row = reinterpret_cast<const float4 *>(rows + x * K);
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const float4 a = row[j ^ sw];  // chunk j of the row
                s = fmaf(a.x, wa[4 * j], fmaf(a.y, wa[4 * j + 1], fmaf(a.z, wa[4 * j + 2], fmaf(a.w, wa[4 * j + 3], s))));
            }
            out[i] = vmax == kNegInf ? kNegInf : T * logf(s) + vmax + tmax;
        }
        o = make_float4(out[0], out[1], out[2], out[3]);
    } else {
        reinterpret_cast<float4 *>(xs)[q] = v;
        __syncwarp();
        float va[K];
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            const float4 a = reinterpret_cast<const float4 *>(xs)[j];
            va[4 * j] = a.x; va[4 * j + 1] = a.y; va[4 * j + 2] = a.z; va[4 * j + 3] = a.w;
        }
        __syncwarp();
        float out[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = 4 * q + i;
            float z[K];
#pragma unroll
            for (int y = 0; y < K; ++y) z[y] = rows[qtab_index<K>(x, y)] + va[y];
            out[i] = lse_row<K, MAXP>(z, T, invT);
        }
        o = make_float4(out[0], out[1], out[2], out[3]);
    }
    return o;
}

template <int K, bool MAXP, bool MS = false>
__global__ void __launch_bounds__(256, 4)
k_pair_quad(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
            const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
            float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    static_assert(K == 8 || K == 16, "four states per lane, K / 4 lanes per factor");
    constexpr int L = K / 4;
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    __shared__ float tab[K * K];                   // phi, row-major (the rare path)
    __shared__ __align__(16) float rows0[K * K];   // E (linear) or phi, rows swizzled (qtab_index)
    __shared__ __align__(16) float rows1[K * K];   // E^T or phi^T
    __shared__ __align__(16) float xchg[256 * 4];
    __shared__ float tinfo[2];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;  // the whole block
    const int n_fac = __ldg(&S->n_fac), pot_base = __ldg(&S->pot_base);
    // the group's shared table (quad groups are planned for shared tables only)
    for (int i = threadIdx.x; i < K * K; i += blockDim.x) tab[i] = __ldg(pot + pot_base + i);
    __syncthreads();
    const bool linear = prepare_linear_table<K, MAXP>(tab, rows0, tinfo, invT);  // rows0 = E, unpadded
    // E (or phi) and its transpose in the swizzled layout (blocks of at least 64 threads)
    {
        constexpr int kPer = (K * K + 63) / 64;
        float e[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * blockDim.x;
            e[k] = i < K * K ? (linear ? rows0[i] : tab[i]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * blockDim.x;
            if (i < K * K) {
                const int r = i / K, c = i % K;
                rows0[qtab_index<K>(r, c)] = e[k];
                rows1[qtab_index<K>(c, r)] = e[k];
            }
        }
        __syncthreads();
    }
    const float tmax = linear ? tinfo[0] : 0.f;
    const int q = threadIdx.x & (L - 1);
    const int fi = (blockIdx.x - __ldg(&S->block_begin)) * (blockDim.x / L) + (threadIdx.x / L);
    const bool valid = fi < n_fac;
    const int f = valid ? fi : n_fac - 1;  // idle lanes shadow the last factor, store nothing
    const int e = __ldg(&S->edge_base) + 2 * f;
    const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
    const int vs0 = __ldg(G.edge_vs + e), vs1 = __ldg(G.edge_vs + e + 1);
    const float4 mo0 = ld4(m_old + es0 + 4 * q, true);
    const float4 mo1 = ld4(m_old + es1 + 4 * q, true);
    const bool rare_lane = (vs0 < 0) | (vs1 < 0) | needs_exact(mo0.x) | needs_exact(mo0.y) | needs_exact(mo0.z) |
                           needs_exact(mo0.w) | needs_exact(mo1.x) | needs_exact(mo1.y) | needs_exact(mo1.z) |
                           needs_exact(mo1.w);
    const unsigned lane = threadIdx.x & 31;
    const unsigned gbits = ((1u << L) - 1u) << (lane & ~(unsigned)(L - 1));
    const bool rare = (__ballot_sync(0xffffffffu, rare_lane) & gbits) != 0u;
    float *xs = xchg + (threadIdx.x & ~(L - 1)) * 4;
    // the common path runs on every lane (the exchanges are warp-synchronous); a rare
    // group's results are discarded
    const float4 b1 = ld4(b + max(vs1, 0) + 4 * q, false);
    float4 v = make_float4(b1.x - mo1.x, b1.y - mo1.y, b1.z - mo1.z, b1.w - mo1.w);
    float4 o0 = quad_dir<K, MAXP>(v, linear, rows0, xs, q, tmax, T, invT);
    const float4 b0 = ld4(b + max(vs0, 0) + 4 * q, false);
    v = make_float4(b0.x - mo0.x, b0.y - mo0.y, b0.z - mo0.z, b0.w - mo0.w);
    float4 o1 = quad_dir<K, MAXP>(v, linear, rows1, xs, q, tmax, T, invT);
    const bool lead = q == 0 && valid && !rare;
    quad_normalise<L>(o0, G.flags, lead);
    quad_normalise<L>(o1, G.flags, lead);
    if (damping != 0.f) {
        const float w = 1.f - damping;
        o0 = make_float4(damping * mo0.x + w * o0.x, damping * mo0.y + w * o0.y, damping * mo0.z + w * o0.z,
                         damping * mo0.w + w * o0.w);
        o1 = make_float4(damping * mo1.x + w * o1.x, damping * mo1.y + w * o1.y, damping * mo1.z + w * o1.z,
                         damping * mo1.w + w * o1.w);
    }
    quad_normalise<L>(o0, G.flags, lead);
    quad_normalise<L>(o1, G.flags, lead);
    if (valid && !rare) {
        st4(m_new + es0 + 4 * q, o0);
        st4(m_new + es1 + 4 * q, o1);
    }
    if (valid && rare && q == 0)
        pair_factor_rare<K, MAXP>(G, tab, pot + pot_base, b, ev, m_old, m_new, vs0, vs1, es0, es1, T, invT, damping);
}

// =====================================================================================
// Factor pass: any listed-configuration factor, thread per factor
// =====================================================================================

template <bool MAXP, bool MS = false>
__global__ void __launch_bounds__(128)
k_enum_generic(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
               const float *__restrict__ b, const float *__restrict__ ev,
               const float *__restrict__ m_old, float *__restrict__ m_new, float T, float invT,
               float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= __ldg(&S->n_fac)) return;
    const int a = __ldg(&S->arity), nc = __ldg(&S->n_cfg), ksum = __ldg(&S->es_per_fac);
    int Kj[kMaxArity], Ko[kMaxArity];
    for (int j = 0; j < a; ++j) {
        Kj[j] = __ldg(&S->K[j]);
        Ko[j] = __ldg(&S->Koff[j]);
    }
    const int es_f = __ldg(&S->es_base) + f * ksum;
    const int e_f = __ldg(&S->edge_base) + f * a;
    float v2f[kMaxStateSum], mo[kMaxStateSum], am[kMaxStateSum], as[kMaxStateSum];
    for (int j = 0; j < a; ++j) {
        const int vs = __ldg(G.edge_vs + e_f + j);
        const int es = es_f + Ko[j];
        float2 hmx = make_float2(-CUDART_INF_F, 0.f);
        bool exact = false;
        const bool lo = G.b_lo != nullptr && Kj[j] > 16;  // a variable of the warp pass
        for (int x = 0; x < Kj[j]; ++x) {
            const float mv = __ldg(m_old + es + x);
            mo[Ko[j] + x] = mv;
            exact |= lo ? !isfinite(mv) : needs_exact(mv);
        }
        if (vs < 0)
            for (int x = 0; x < Kj[j]; ++x) {
                const float2 q = hd_pair(G, vs, x, mo[Ko[j] + x]);
                if (x == 0 || hd_gt(q, hmx)) hmx = q;
            }
        if (vs < 0) {
            for (int x = 0; x < Kj[j]; ++x)
                v2f[Ko[j] + x] =
                    hmx.x == -CUDART_INF_F ? -CUDART_INF_F : hd_rel(hd_pair(G, vs, x, mo[Ko[j] + x]), hmx);
        } else if (exact) {
            v2f_slow_edge(G, ev, m_old, vs, es, Kj[j], v2f + Ko[j]);
        } else if (lo) {
            for (int x = 0; x < Kj[j]; ++x)
                v2f[Ko[j] + x] = (__ldg(b + vs + x) - mo[Ko[j] + x]) + __ldg(G.b_lo + vs + x);
        } else {
            for (int x = 0; x < Kj[j]; ++x) v2f[Ko[j] + x] = __ldg(b + vs + x) - mo[Ko[j] + x];
        }
    }
    for (int i = 0; i < ksum; ++i) {
        am[i] = kNegInf;
        as[i] = 0.f;
    }
    const uint8_t *cfg = G.cfg_pool + __ldg(&S->cfg_base);
    const float *phi = pot + __ldg(&S->pot_base) + (__ldg(&S->shared) ? 0 : (size_t)f * nc);
    for (int c = 0; c < nc; ++c) {
        const float ph = __ldg(phi + c);
        const uint8_t *cc = cfg + c * a;
        for (int i = 0; i < a; ++i) {
            float val = ph;
            for (int j = 0; j < a; ++j)
                if (j != i) val += v2f[Ko[j] + __ldg(cc + j)];
            const int idx = Ko[i] + __ldg(cc + i);
            if (MAXP) {
                am[idx] = fmaxf(am[idx], val);
            } else if (val > am[idx]) {
                as[idx] = as[idx] * expf((am[idx] - val) * invT) + 1.f;
                am[idx] = val;
            } else if (val > kNegInf) {
                as[idx] += expf((val - am[idx]) * invT);
            }
        }
    }
    const float w = 1.f - damping;
    for (int j = 0; j < a; ++j) {
        float *t = am + Ko[j];
        const int K = Kj[j];
        if (!MAXP)
            for (int x = 0; x < K; ++x)
                if (t[x] != kNegInf) t[x] += T * logf(as[Ko[j] + x]);
        normalise_rt(t, K, G.flags);
        if (damping != 0.f)
            for (int x = 0; x < K; ++x) t[x] = damping * mo[Ko[j] + x] + w * t[x];
        normalise_rt(t, K, G.flags);
        for (int x = 0; x < K; ++x) m_new[es_f + Ko[j] + x] = t[x];
    }
}

// =====================================================================================
// Factor pass: large listed-configuration factors, a team per factor
// =====================================================================================

// Factors given by a long list of valid configurations or with many states (Sec. 5.2:
// the irregular pairwise factors of RCN are given this way), beyond the thread-per-factor
// kernel's kMaxStateSum. A block takes fpb consecutive factors of one group; a team -- a
// warp when the state sum is at most kEnumWarpStateSum (so a 256-thread block has 8
// factors in flight and no block-wide barrier), else the whole block -- takes one factor
// at a time. The group's table (each configuration's states, the configurations listed
// by output edge-state, a shared log-potential table) is staged once per block in shared
// memory when it fits (table_bytes > 0), else read in place. Per factor:
//   (1) a thread per edge-state writes b - m (plus b_lo for variables with more than 16
//       states) to the team's shared arrays, keeping m for step 3; an edge with an entry
//       that needs the explicit sums, or of a high-degree variable, is redone by a warp;
//   (2) `lanes` threads per output edge-state (j, x) walk the configurations with state
//       x at neighbour j; each value is the log-potential plus the other neighbours'
//       variable-to-factor values, reduced by max (T = 0) or a running log-sum-exp
//       (T > 0); the lanes of an output combine by shuffles; a pairwise group's list
//       entries carry the other neighbour's state offset with the configuration id;
//   (3) a warp per edge normalises, damps and normalises the edge's message.
// Every output sums its terms in neighbour order; a group with `ordered` set (one lane per
// output) reduces its configurations in ascending order, as the thread-per-factor kernel
// does, and the two give the same bits; otherwise T > 0 differs by rounding.
// v2f_slow_edge for the edge of variable v, the states spread over the lanes of a warp
// (same sums, same bits).
__device__ __noinline__ void v2f_slow_edge_warp(const DevGraph G, const float *__restrict__ ev,
                                                const float *__restrict__ m, int v, int vs, int es, int K,
                                                float *out, int lane) {
    const int k0 = G.vin_off[v], k1 = G.vin_off[v + 1];
    for (int x = lane; x < K; x += 32) {
        FF s = ff_make(ev[vs + x]);
        for (int k = k0; k < k1; ++k) {
            const int e2 = G.vin_es[k];
            if (e2 != es) s = ff_add(s, m[e2 + x]);
        }
        out[x] = s.hi + s.lo;
    }
}

// A barrier over a factor's team: the warp, or the whole block.
__device__ __forceinline__ void team_barrier(bool wteam) {
    if (wteam) __syncwarp();
    else __syncthreads();
}

// Step (1) of the team kernels (k_enum_block, k_adj_block): the factor's variable-to-factor
// values into v2f[ksum] (and its stored messages into smo[ksum] if not null), as
// k_enum_generic forms them: b - m by a thread per edge-state (plus the belief residual
// for variables of more than 16 states); an edge with an entry that needs the explicit
// leave-one-out sums, or of a high-degree variable, is then redone by a warp. fix[a]:
// the team's flags. Ends with a team barrier.
__device__ __forceinline__ void enum_team_v2f(const DevGraph &G, const float *__restrict__ b,
                                              const float *__restrict__ ev, const float *__restrict__ m_old,
                                              int e_f, int es_f, int a, int ksum, const int *sK, const int *sKo,
                                              float *v2f, float *smo, int *fix, bool wteam, int trank, int tsize,
                                              int ej0, int ejs, int lane) {
    if (trank < a) fix[trank] = 0;
    team_barrier(wteam);
    for (int t = trank; t < ksum; t += tsize) {
        int j = 0;
        for (int k = 1; k < a; ++k)
            if (t >= sKo[k]) j = k;
        const int vs = __ldg(G.edge_vs + e_f + j);
        const float mo = __ldg(m_old + es_f + t);
        if (smo) smo[t] = mo;
        const bool lo = G.b_lo != nullptr && sK[j] > 16;  // (as in k_enum_generic)
        if (vs < 0 || (lo ? !isfinite(mo) : needs_exact(mo))) fix[j] = 1;  // benign race: all write 1
        else if (lo) v2f[t] = (__ldg(b + vs + t - sKo[j]) - mo) + __ldg(G.b_lo + vs + t - sKo[j]);
        else v2f[t] = __ldg(b + vs + t - sKo[j]) - mo;
    }
    team_barrier(wteam);
    for (int j = ej0; j < a; j += ejs) {
        if (!fix[j]) continue;  // warp-uniform
        const int vs = __ldg(G.edge_vs + e_f + j), es = es_f + sKo[j], K = sK[j];
        float *vj = v2f + sKo[j];
        if (vs >= 0) {
            v2f_slow_edge_warp(G, ev, m_old, __ldg(G.edge_var + e_f + j), vs, es, K, vj, lane);
            continue;
        }
        // the largest state (first of equals), then every state relative to it
        float2 hmx = make_float2(-CUDART_INF_F, 0.f);
        int hx = K;
        for (int x = lane; x < K; x += 32) {
            const float2 q = hd_pair(G, vs, x, __ldg(m_old + es + x));
            if (hx == K || hd_gt(q, hmx)) {
                hmx = q;
                hx = x;
            }
        }
        for (int d = 16; d > 0; d >>= 1) {
            const float2 q = make_float2(__shfl_xor_sync(0xffffffffu, hmx.x, d),
                                         __shfl_xor_sync(0xffffffffu, hmx.y, d));
            const int qx = __shfl_xor_sync(0xffffffffu, hx, d);
            const bool take = qx < K && (hx == K || hd_gt(q, hmx) || (!hd_gt(hmx, q) && qx < hx));
            if (take) {
                hmx = q;
                hx = qx;
            }
        }
        for (int x = lane; x < K; x += 32)
            vj[x] = hmx.x == -CUDART_INF_F ? -CUDART_INF_F : hd_rel(hd_pair(G, vs, x, __ldg(m_old + es + x)), hmx);
    }
    team_barrier(wteam);
}

// One output of a packed pairwise list walked by lane gl of its L lanes: entries
// i0, i0 + L, .. < i1, each (configuration << 11) | the other neighbour's state offset,
// scored phi(configuration) + v2f(other state). STAGED: the entries come as
// (entry, log-potential) pairs (fl), so one 8-byte shared read replaces the entry read
// and the dependent log-potential gather. Same order of operations as the unstaged walk.
template <bool MAXP, bool STAGED>
__device__ __forceinline__ void enum_packed_output(const int2 *fl, const int32_t *lst, const float *phi,
                                                   const float *v2f, int i, int i1, int L, int ordered, float invT,
                                                   float &mx, float &sm) {
    auto score = [&](int k) {
        if constexpr (STAGED) {
            const int2 p = fl[k];
            return __int_as_float(p.y) + v2f[p.x & 2047];
        } else {
            const int e = lst[k];
            return phi[e >> 11] + v2f[e & 2047];
        }
    };
    if (MAXP) {
        float m1 = kNegInf, m2 = kNegInf, m3 = kNegInf;
        for (; i + 3 * L < i1; i += 4 * L) {
            mx = fmaxf(mx, score(i));
            m1 = fmaxf(m1, score(i + L));
            m2 = fmaxf(m2, score(i + 2 * L));
            m3 = fmaxf(m3, score(i + 3 * L));
        }
        mx = fmaxf(fmaxf(mx, m1), fmaxf(m2, m3));
    } else if (!ordered) {
        float mb = kNegInf, sb = 0.f;
        for (; i + L < i1; i += 2 * L) {
            const float va = score(i), vb = score(i + L);
            if (va > mx) {
                sm = sm * expf((mx - va) * invT) + 1.f;
                mx = va;
            } else if (va > kNegInf) {
                sm += expf((va - mx) * invT);
            }
            if (vb > mb) {
                sb = sb * expf((mb - vb) * invT) + 1.f;
                mb = vb;
            } else if (vb > kNegInf) {
                sb += expf((vb - mb) * invT);
            }
        }
        const float mn = fmaxf(mx, mb);
        if (mn != kNegInf) {
            sm = (mx == kNegInf ? 0.f : sm * expf((mx - mn) * invT)) + (mb == kNegInf ? 0.f : sb * expf((mb - mn) * invT));
            mx = mn;
        }
    }
    for (; i < i1; i += L) {
        const float val = score(i);
        if (MAXP) {
            mx = fmaxf(mx, val);
        } else if (val > mx) {
            sm = sm * expf((mx - val) * invT) + 1.f;
            mx = val;
        } else if (val > kNegInf) {
            sm += expf((val - mx) * invT);
        }
    }
}

template <bool MAXP, bool MS = false>
__global__ void __launch_bounds__(kEnumBlockThreads)
k_enum_block(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
             const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
             float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        pot += smp * G.s_pot;
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    extern __shared__ __align__(16) unsigned char eb_smem[];
    __shared__ int sK[kMaxArity], sKo[kMaxArity];
    __shared__ int s_fix[kEnumBlockThreads / 32][kMaxArity];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;  // the whole block
    const int a = __ldg(&S->arity), nc = __ldg(&S->n_cfg), ksum = __ldg(&S->es_per_fac);
    const int fpb = __ldg(&S->fpb), L = __ldg(&S->lanes), tb = __ldg(&S->table_bytes);
    const int n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared), packed = __ldg(&S->packed);
    const int ordered = __ldg(&S->ordered);
    const int f0 = (blockIdx.x - __ldg(&S->block_begin)) * fpb;
    const int f1 = min(n_fac, f0 + fpb);
    if (threadIdx.x < a) {
        sK[threadIdx.x] = __ldg(&S->K[threadIdx.x]);
        sKo[threadIdx.x] = __ldg(&S->Koff[threadIdx.x]);
    }
    // teams (uniform over the block)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const bool wteam = ksum <= kEnumWarpStateSum;
    const int tsize = wteam ? 32 : (int)blockDim.x, trank = wteam ? lane : (int)threadIdx.x;
    const int team = wteam ? warp : 0, n_teams = wteam ? nw : 1;
    const int ej0 = wteam ? 0 : warp, ejs = wteam ? 1 : nw;  // the edges a warp takes
    float *v2f = reinterpret_cast<float *>(eb_smem) + (size_t)team * 3 * ksum;  // [ksum]
    float *out = v2f + ksum;                                                  // [ksum]
    float *smo = out + ksum;                                                  // [ksum]
    const int cfg_bytes = (nc * a + 15) & ~15;
    const int ob = (ksum + 1 + 3) & ~3;  // offsets block, then the lists
    const int bs_len = (ob + a * nc + 3) & ~3;
    const uint8_t *cfg = G.cfg_pool + __ldg(&S->cfg_base);
    const int32_t *bs = G.bs_pool + __ldg(&S->bs_base);
    const float *phi_g = pot + __ldg(&S->pot_base);
    const float *phi_tab = phi_g;
    const int2 *flst = nullptr;  // staged (entry, log-potential) pairs of a packed shared list
    if (tb > 0 && shared && packed) {
        // packed pairwise lists with a shared table: the offsets, then each list entry
        // beside its configuration's log-potential (one 8-byte read per entry); the
        // configuration table and the log-potentials are not read in this form
        unsigned char *t = eb_smem + ((12 * ksum * n_teams + 15) & ~15);
        int32_t *tbs = reinterpret_cast<int32_t *>(t);
        for (int i = threadIdx.x; i < ob; i += blockDim.x) tbs[i] = __ldg(bs + i);
        int2 *fl = reinterpret_cast<int2 *>(t + 4 * ob);  // 4 ob is a multiple of 16
        for (int i = threadIdx.x; i < a * nc; i += blockDim.x) {
            const int e = __ldg(bs + ob + i);
            fl[i] = make_int2(e, __float_as_int(__ldg(phi_g + (e >> 11))));
        }
        flst = fl;
        bs = tbs;
    } else if (tb > 0) {  // 16-byte aligned sources (pool layout) and destinations
        unsigned char *t = eb_smem + ((12 * ksum * n_teams + 15) & ~15);
        const uint4 *c_src = reinterpret_cast<const uint4 *>(cfg);
        uint4 *c_dst = reinterpret_cast<uint4 *>(t);
        for (int i = threadIdx.x; i < cfg_bytes / 16; i += blockDim.x) c_dst[i] = __ldg(c_src + i);
        int32_t *tbs = reinterpret_cast<int32_t *>(t + cfg_bytes);
        const int4 *b_src = reinterpret_cast<const int4 *>(bs);
        int4 *b_dst = reinterpret_cast<int4 *>(tbs);
        for (int i = threadIdx.x; i < bs_len / 4; i += blockDim.x) b_dst[i] = __ldg(b_src + i);
        if (shared) {
            float *tphi = reinterpret_cast<float *>(tbs + bs_len);
            for (int i = threadIdx.x; i < nc; i += blockDim.x) tphi[i] = __ldg(phi_g + i);
            phi_tab = tphi;
        }
        cfg = t;
        bs = tbs;
    }
    __syncthreads();  // the last block-wide barrier when teams are warps
    const int ng = tsize / L, gi = trank / L, gl = trank - gi * L;
    const int32_t *lst = bs + ob;
    const float w = 1.f - damping;
    for (int f = f0 + team; f < f1; f += n_teams) {
        const int es_f = __ldg(&S->es_base) + f * ksum;
        const int e_f = __ldg(&S->edge_base) + f * a;
        // (1) variable-to-factor values
        enum_team_v2f(G, b, ev, m_old, e_f, es_f, a, ksum, sK, sKo, v2f, smo, s_fix[team], wteam, trank, tsize,
                      ej0, ejs, lane);
        // (2) every output edge-state over its configurations
        const float *phi = shared ? phi_tab : phi_g + (size_t)f * nc;
        for (int base = 0; base < ksum; base += ng) {
            const int o = base + gi;
            float mx = kNegInf, sm = 0.f;
            if (o < ksum && flst != nullptr) {
                // staged pairs: one 8-byte read gives the entry and its log-potential
                enum_packed_output<MAXP, true>(flst, lst, phi, v2f, bs[o] + gl, bs[o + 1], L, ordered, invT, mx, sm);
            } else if (o < ksum && packed) {
                // pairwise: entry = (configuration << 11) | the other neighbour's
                // state offset; at T = 0 four independent max chains; at T > 0 two
                // log-sum-exp chains unless the group keeps the ascending order
                const int i1 = bs[o + 1];
                int i = bs[o] + gl;
                if (MAXP) {
                    float m1 = kNegInf, m2 = kNegInf, m3 = kNegInf;
                    for (; i + 3 * L < i1; i += 4 * L) {
                        const int e0 = lst[i], e1 = lst[i + L], e2 = lst[i + 2 * L], e3 = lst[i + 3 * L];
                        mx = fmaxf(mx, phi[e0 >> 11] + v2f[e0 & 2047]);
                        m1 = fmaxf(m1, phi[e1 >> 11] + v2f[e1 & 2047]);
                        m2 = fmaxf(m2, phi[e2 >> 11] + v2f[e2 & 2047]);
                        m3 = fmaxf(m3, phi[e3 >> 11] + v2f[e3 & 2047]);
                    }
                    mx = fmaxf(fmaxf(mx, m1), fmaxf(m2, m3));
                } else if (!ordered) {
                    float mb = kNegInf, sb = 0.f;
                    for (; i + L < i1; i += 2 * L) {
                        const int e0 = lst[i], e1 = lst[i + L];
                        const float va = phi[e0 >> 11] + v2f[e0 & 2047], vb = phi[e1 >> 11] + v2f[e1 & 2047];
                        if (va > mx) {
                            sm = sm * expf((mx - va) * invT) + 1.f;
                            mx = va;
                        } else if (va > kNegInf) {
                            sm += expf((va - mx) * invT);
                        }
                        if (vb > mb) {
                            sb = sb * expf((mb - vb) * invT) + 1.f;
                            mb = vb;
                        } else if (vb > kNegInf) {
                            sb += expf((vb - mb) * invT);
                        }
                    }
                    const float mn = fmaxf(mx, mb);
                    if (mn != kNegInf) {
                        sm = (mx == kNegInf ? 0.f : sm * expf((mx - mn) * invT)) +
                             (mb == kNegInf ? 0.f : sb * expf((mb - mn) * invT));
                        mx = mn;
                    }
                }
                for (; i < i1; i += L) {
                    const int e = lst[i];
                    const float val = phi[e >> 11] + v2f[e & 2047];
                    if (MAXP) {
                        mx = fmaxf(mx, val);
                    } else if (val > mx) {
                        sm = sm * expf((mx - val) * invT) + 1.f;
                        mx = val;
                    } else if (val > kNegInf) {
                        sm += expf((val - mx) * invT);
                    }
                }
            } else if (o < ksum) {
                int j = 0;
                for (int k = 1; k < a; ++k)
                    if (o >= sKo[k]) j = k;
                const int i1 = bs[o + 1];
                for (int i = bs[o] + gl; i < i1; i += L) {
                    const int c = lst[i];
                    const uint8_t *cc = cfg + c * a;
                    float val = phi[c];
                    for (int k = 0; k < a; ++k)
                        if (k != j) val += v2f[sKo[k] + cc[k]];
                    if (MAXP) {
                        mx = fmaxf(mx, val);
                    } else if (val > mx) {
                        sm = sm * expf((mx - val) * invT) + 1.f;
                        mx = val;
                    } else if (val > kNegInf) {
                        sm += expf((val - mx) * invT);
                    }
                }
            }
            for (int d = 1; d < L; d <<= 1) {  // L a power of two; whole warps take part
                const float m2 = __shfl_xor_sync(0xffffffffu, mx, d);
                if (MAXP) {
                    mx = fmaxf(mx, m2);
                } else {
                    const float s2 = __shfl_xor_sync(0xffffffffu, sm, d);
                    const float mn = fmaxf(mx, m2);
                    if (mn != kNegInf) {
                        sm = (mx == kNegInf ? 0.f : sm * expf((mx - mn) * invT)) +
                             (m2 == kNegInf ? 0.f : s2 * expf((m2 - mn) * invT));
                        mx = mn;
                    }
                }
            }
            if (o < ksum && gl == 0) out[o] = (MAXP || mx == kNegInf) ? mx : mx + T * logf(sm);
        }
        team_barrier(wteam);
        // (3) normalise, damp, normalise; a warp per edge, up to 8 states per lane
        for (int j = ej0; j < a; j += ejs) {
            const int K = sK[j], es = es_f + sKo[j];
            const float *t = out + sKo[j], *mo = smo + sKo[j];
            float v[kMaxStates / 32];
            float mx = kNegInf;
#pragma unroll
            for (int r = 0; r < kMaxStates / 32; ++r) {
                const int x = lane + 32 * r;
                v[r] = x < K ? t[x] : kNegInf;
                if (v[r] > mx) mx = v[r];
            }
            for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
            if (mx == kNegInf && lane == 0) atomicOr(G.flags, kFlagContradiction);
            float mx2 = kNegInf;
#pragma unroll
            for (int r = 0; r < kMaxStates / 32; ++r) {
                const int x = lane + 32 * r;
                if (x < K) {
                    float y = mx == kNegInf ? 0.f : v[r] - mx;
                    if (damping != 0.f) y = damping * mo[x] + w * y;
                    v[r] = y;
                    if (y > mx2) mx2 = y;
                }
            }
            for (int d = 16; d > 0; d >>= 1) mx2 = fmaxf(mx2, __shfl_xor_sync(0xffffffffu, mx2, d));
            if (mx2 == kNegInf && lane == 0) atomicOr(G.flags, kFlagContradiction);
#pragma unroll
            for (int r = 0; r < kMaxStates / 32; ++r) {
                const int x = lane + 32 * r;
                if (x < K) m_new[es + x] = mx2 == kNegInf ? 0.f : v[r] - mx2;
            }
        }
    }
}

// =====================================================================================
// Factor pass: logical OR / AND
// =====================================================================================

// Writes the damped, normalised message for one binary edge from its outgoing
// log-odds `o` (already in the OR frame times sgn).
__device__ __forceinline__ void write_logic_edge(float o, const float2 mo, float *m_new, int es,
                                                 float damping, uint32_t *flags) {
    float t[2], old[2] = {mo.x, mo.y};
    if (o >= 0.f) {
        t[0] = -o;
        t[1] = 0.f;
    } else {
        t[0] = 0.f;
        t[1] = o;
    }
    finish_k<2>(t, old, damping, flags);
    float *q = m_new + es;
    if ((reinterpret_cast<uintptr_t>(q) & 7u) == 0) {
        *reinterpret_cast<float2 *>(q) = make_float2(t[0], t[1]);
    } else {
        q[0] = t[0];
        q[1] = t[1];
    }
}

// Two consecutive floats: one 8-byte load when the address allows it (edge-states of
// binary edges start on even offsets when every edge before them is binary), else two.
__device__ __forceinline__ float2 ld2(const float *p) {
    if ((reinterpret_cast<uintptr_t>(p) & 7u) == 0) return __ldg(reinterpret_cast<const float2 *>(p));
    return make_float2(__ldg(p), __ldg(p + 1));
}

// Incoming log-odds of one edge (times sgn) and its stored message.
__device__ __forceinline__ float edge_logodds(const DevGraph &G, const float *ev, const float *b,
                                              const float *m_old, int e, int es, float sgn,
                                              float2 &mo) {
    const int vs = __ldg(G.edge_vs + e);
    mo = ld2(m_old + es);
    float a0, a1;
    if (vs < 0) {
        float t[2];
        const float m2[2] = {mo.x, mo.y};
        hd_v2f<2>(G, vs, m2, t);
        a0 = t[0];
        a1 = t[1];
    } else if (needs_exact(mo.x) || needs_exact(mo.y)) {
        if (G.b_lo != nullptr && isfinite(mo.x) && isfinite(mo.y)) {
            // the variable pass saw this large entry and wrote the belief residuals:
            // b - m without the cancellation, rounded twice
            const float2 bb = ld2(b + vs), bl = ld2(G.b_lo + vs);
            a0 = (bb.x - mo.x) + bl.x;
            a1 = (bb.y - mo.y) + bl.y;
        } else {
            float t[2];
            v2f_slow_edge(G, ev, m_old, vs, es, 2, t);
            a0 = t[0];
            a1 = t[1];
        }
    } else {
        const float2 bb = ld2(b + vs);
        a0 = bb.x - mo.x;
        a1 = bb.y - mo.y;
    }
    return sgn * log_odds(a0, a1);
}

// Thread per factor, fan-in <= F (F = kLogicSmallFan, or 2 for launches whose groups
// have at most two parents, which keeps fewer registers); leave-one-out sums written out
// directly.
template <bool MAXP, bool MS = false, int F = kLogicSmallFan>
__global__ void __launch_bounds__(256)
k_logic_small(DevGraph G, const LogicSeg *__restrict__ segs, int n_seg, const float *__restrict__ b,
              const float *__restrict__ ev, const float *__restrict__ m_old,
              float *__restrict__ m_new, float T, float invT, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    const LogicSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= __ldg(&S->n_fac)) return;
    const int *po = G.paroff_pool + __ldg(&S->paroff_base);
    const int p0 = __ldg(po + f), n = __ldg(po + f + 1) - p0;
    const int edge_base = __ldg(&S->edge_base), es_base = __ldg(&S->es_base);
    const int e0 = edge_base + p0 + f;
    const float sgn = __ldg(&S->kind) == PGM_LOGIC_AND ? -1.f : 1.f;
    // parents in unrolled slots (j < n valid) and the child apart, so that every array
    // index is a constant and the values stay in registers
    float x[F];
    float2 mo[F], moc;
#pragma unroll
    for (int k = 0; k < F; ++k) {
        x[k] = 0.f;
        mo[k] = make_float2(0.f, 0.f);
        if (k < n) {
            const int e = e0 + k;
            x[k] = edge_logodds(G, ev, b, m_old, e, es_base + 2 * (e - edge_base), sgn, mo[k]);
        }
    }
    const float xc = edge_logodds(G, ev, b, m_old, e0 + n, es_base + 2 * (e0 + n - edge_base), sgn, moc);
    float out[F], outc;
    if (__ldg(&S->kind) == PGM_LOGIC_XOR) {  // sgn = +1
        bool pos_all = xc > 0.f;  // parity of all members' positive log-odds
#pragma unroll
        for (int j = 0; j < F; ++j)
            if (j < n) pos_all ^= x[j] > 0.f;
        if (MAXP) {
            float mall = CUDART_INF_F;  // smallest |x| over the parents
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (j < n) mall = fminf(mall, fabsf(x[j]));
            outc = xor_out_max(mall, pos_all ^ (xc > 0.f));
#pragma unroll
            for (int i = 0; i < F; ++i) {
                float mn = fabsf(xc);
#pragma unroll
                for (int j = 0; j < F; ++j)
                    if (j < n && j != i) mn = fminf(mn, fabsf(x[j]));
                out[i] = xor_out_max(mn, pos_all ^ (x[i] > 0.f));
            }
        } else {
            const double Td = T;
            double l[F];
#pragma unroll
            for (int j = 0; j < F; ++j) l[j] = j < n ? xor_log_u((double)x[j] / Td) : -CUDART_INF;
            const double lc = xor_log_u((double)xc / Td);
            double all = -CUDART_INF;
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (j < n) all = lse2_d(all, l[j]);
            outc = xor_out_soft(all, pos_all ^ (xc > 0.f), Td);
#pragma unroll
            for (int i = 0; i < F; ++i) {
                // the others as prefix (parents before i, ascending) and suffix (the
                // child, then the parents after i, descending)
                double pre = -CUDART_INF, suf = lc;
#pragma unroll
                for (int j = 0; j < F; ++j)
                    if (j < i) pre = lse2_d(pre, l[j]);
#pragma unroll
                for (int j = F - 1; j >= 0; --j)
                    if (j < n && j > i) suf = lse2_d(suf, l[j]);
                out[i] = xor_out_soft(lse2_d(pre, suf), pos_all ^ (x[i] > 0.f), Td);
            }
        }
    } else if (MAXP) {
        float A = 0.f, Mall = kNegInf;
#pragma unroll
        for (int j = 0; j < F; ++j)
            if (j < n) {
                A += fmaxf(x[j], 0.f);
                Mall = fmaxf(Mall, x[j]);
            }
        outc = A + (Mall < 0.f ? Mall : 0.f);
#pragma unroll
        for (int i = 0; i < F; ++i) {
            float Si = 0.f, Mi = kNegInf;
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (j < n && j != i) {
                    Si += fmaxf(x[j], 0.f);
                    Mi = fmaxf(Mi, x[j]);
                }
            out[i] = or_parent_max(Si, Mi, xc);
        }
    } else {
        const double Td = T;
        double t[F];
        double all = -CUDART_INF;
#pragma unroll
        for (int j = 0; j < F; ++j) {
            t[j] = (j >= n || x[j] == kNegInf) ? -CUDART_INF : log_softplus_d((double)x[j] / Td);
            if (j < n) all = lse2_d(all, t[j]);
        }
        outc = (float)(Td * log_expm1_from_log_d(all));
#pragma unroll
        for (int i = 0; i < F; ++i) {
            double li = -CUDART_INF;
#pragma unroll
            for (int j = 0; j < F; ++j)
                if (j < n && j != i) li = lse2_d(li, t[j]);
            out[i] = or_parent_soft(li, xc, Td);
        }
    }
#pragma unroll
    for (int k = 0; k < F; ++k)
        if (k < n) {
            const int e = e0 + k;
            write_logic_edge(sgn * out[k], mo[k], m_new, es_base + 2 * (e - edge_base), damping, G.flags);
        }
    write_logic_edge(sgn * outc, moc, m_new, es_base + 2 * (e0 + n - edge_base), damping, G.flags);
}

// Scan element of the warp OR / AND kernel. T = 0: (a, b) = (sum of max(x_j, 0),
// max x_j) in FP32. T > 0: a single FP64 log-sum (LSE of log s(x_j / T)) held in the
// bits of (a, b).
struct ScanEl {
    float a, b;
};

__device__ __forceinline__ double el_d(ScanEl e) {
    return __hiloint2double(__float_as_int(e.a), __float_as_int(e.b));
}
__device__ __forceinline__ ScanEl d_el(double d) {
    return ScanEl{__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d))};
}

// XOR: T = 0, a = smallest |x_j| (b unused); T > 0, the FP64 LSE of xor_log_u(x_j / T).
template <bool MAXP, bool XOR = false>
__device__ __forceinline__ ScanEl scan_ident() {
    if (XOR && MAXP) return ScanEl{CUDART_INF_F, 0.f};
    return MAXP ? ScanEl{0.f, kNegInf} : d_el(-CUDART_INF);
}

template <bool MAXP, bool XOR = false>
__device__ __forceinline__ ScanEl scan_comb(ScanEl p, ScanEl q) {
    if (XOR && MAXP) return ScanEl{fminf(p.a, q.a), 0.f};
    if (MAXP) return ScanEl{p.a + q.a, fmaxf(p.b, q.b)};
    return d_el(lse2_d(el_d(p), el_d(q)));
}

template <bool MAXP, bool XOR = false>
__device__ __forceinline__ ScanEl scan_elem(float x, double T) {
    if (XOR) return MAXP ? ScanEl{fabsf(x), 0.f} : d_el(xor_log_u((double)x / T));
    if (MAXP) return ScanEl{fmaxf(x, 0.f), x};
    return d_el(x == kNegInf ? -CUDART_INF : log_softplus_d((double)x / T));
}

template <bool MAXP>
__device__ __forceinline__ ScanEl shfl_up_el(ScanEl v, int d) {
    return ScanEl{__shfl_up_sync(0xffffffffu, v.a, d), __shfl_up_sync(0xffffffffu, v.b, d)};
}
template <bool MAXP>
__device__ __forceinline__ ScanEl shfl_down_el(ScanEl v, int d) {
    return ScanEl{__shfl_down_sync(0xffffffffu, v.a, d), __shfl_down_sync(0xffffffffu, v.b, d)};
}
__device__ __forceinline__ ScanEl shfl_el(ScanEl v, int src) {
    return ScanEl{__shfl_sync(0xffffffffu, v.a, src), __shfl_sync(0xffffffffu, v.b, src)};
}

// One factor of k_logic_warp (XOR: the parity form; the suffix scan starts from the
// child's element, so that the leave-one-out combination of a parent covers the child).
template <bool MAXP, bool XOR>
__device__ __forceinline__ void logic_warp_factor(const DevGraph &G, const float *__restrict__ b,
                                                  const float *__restrict__ ev, const float *__restrict__ m_old,
                                                  float *__restrict__ m_new, float T, float damping, int e0, int n,
                                                  int edge_base, int es_base, float sgn, float *sx, float *spa,
                                                  float *spb, int lane) {
    const ScanEl ident = scan_ident<MAXP, XOR>();
    // child
    float2 moc = make_float2(0.f, 0.f);
    float xc = 0.f;
    if (lane == 0) xc = edge_logodds(G, ev, b, m_old, e0 + n, es_base + 2 * (e0 + n - edge_base), sgn, moc);
    xc = __shfl_sync(0xffffffffu, xc, 0);
    // forward pass: exclusive prefix (XOR: and the parity of the parents' positive log-odds)
    ScanEl carry = ident;
    bool par = false;
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        const bool valid = j < n;
        float xv = 0.f;
        ScanEl v = ident;
        if (valid) {
            float2 mo;
            const int e = e0 + j;
            xv = edge_logodds(G, ev, b, m_old, e, es_base + 2 * (e - edge_base), sgn, mo);
            v = scan_elem<MAXP, XOR>(xv, (double)T);
        }
        if (XOR) par ^= __popc(__ballot_sync(0xffffffffu, valid && xv > 0.f)) & 1;
        ScanEl inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const ScanEl y = shfl_up_el<MAXP>(inc, d);
            if (lane >= d) inc = scan_comb<MAXP, XOR>(y, inc);
        }
        ScanEl exc = shfl_up_el<MAXP>(inc, 1);
        if (lane == 0) exc = ident;
        if (valid) {
            const ScanEl pre = scan_comb<MAXP, XOR>(carry, exc);
            sx[j] = xv;
            spa[j] = pre.a;
            spb[j] = pre.b;
        }
        carry = scan_comb<MAXP, XOR>(carry, shfl_el(inc, 31));
    }
    __syncwarp();
    const bool pos_all = par ^ (xc > 0.f);  // XOR: parity of all members' positive log-odds
    float out_c;
    if (XOR) out_c = MAXP ? xor_out_max(carry.a, par) : xor_out_soft(el_d(carry), par, (double)T);
    else if (MAXP) out_c = carry.a + (carry.b < 0.f ? carry.b : 0.f);
    else out_c = (float)((double)T * log_expm1_from_log_d(el_d(carry)));
    // backward pass: exclusive suffix, outputs
    ScanEl sc = XOR ? scan_elem<MAXP, XOR>(xc, (double)T) : ident;
    for (int base = n > 0 ? ((n - 1) & ~31) : -32; base >= 0; base -= 32) {
        const int j = base + lane;
        const bool valid = j < n;
        const float xv = valid ? sx[j] : 0.f;
        const ScanEl v = valid ? scan_elem<MAXP, XOR>(xv, (double)T) : ident;
        ScanEl inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const ScanEl y = shfl_down_el<MAXP>(inc, d);
            if (lane + d < 32) inc = scan_comb<MAXP, XOR>(inc, y);
        }
        ScanEl exc = shfl_down_el<MAXP>(inc, 1);
        if (lane == 31) exc = ident;
        if (valid) {
            const ScanEl suf = scan_comb<MAXP, XOR>(exc, sc);
            const ScanEl loo = scan_comb<MAXP, XOR>(ScanEl{spa[j], spb[j]}, suf);
            float o;
            if (XOR) {
                const bool odd = pos_all ^ (xv > 0.f);
                o = MAXP ? xor_out_max(loo.a, odd) : xor_out_soft(el_d(loo), odd, (double)T);
            } else {
                o = MAXP ? or_parent_max(loo.a, loo.b, xc) : or_parent_soft(el_d(loo), xc, (double)T);
            }
            const int e = e0 + j;
            const int es = es_base + 2 * (e - edge_base);
            write_logic_edge(sgn * o, ld2(m_old + es), m_new, es, damping, G.flags);
        }
        sc = scan_comb<MAXP, XOR>(sc, shfl_el(inc, 0));
    }
    if (lane == 0) {
        const int e = e0 + n;
        write_logic_edge(sgn * out_c, moc, m_new, es_base + 2 * (e - edge_base), damping, G.flags);
    }
}

// Warp per factor, any fan-in. Leave-one-out sums as exclusive prefix (first pass) and
// exclusive suffix (second pass) warp scans over rounds of 32 parents; the log-odds
// and the prefix of each parent are staged in shared memory (3 floats per parent).
template <bool MAXP, bool MS = false>
__global__ void __launch_bounds__(128)
k_logic_warp(DevGraph G, const LogicSeg *__restrict__ segs, int n_seg, const float *__restrict__ b,
             const float *__restrict__ ev, const float *__restrict__ m_old,
             float *__restrict__ m_new, float T, float invT, float damping, int cap) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    if constexpr (MS) {  // multi-sample launches: this block's sample
        const int64_t smp = sample_select(G);
        b += smp * G.s_vs;
        ev += smp * G.s_vs;
        m_old += smp * G.s_es;
        m_new += smp * G.s_es;
    }
    extern __shared__ float smem[];
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LogicSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    if (member_skip<MAXP>(G, S->member, T, invT, damping)) return;
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * warps + warp;
    if (f >= __ldg(&S->n_fac)) return;
    float *sx = smem + (size_t)warp * 3 * cap;  // log-odds x_j (times sgn)
    float *spa = sx + cap;                       // exclusive prefix, first component
    float *spb = spa + cap;                      // exclusive prefix, second component
    const int *po = G.paroff_pool + __ldg(&S->paroff_base);
    const int p0 = __ldg(po + f), n = __ldg(po + f + 1) - p0;
    const int edge_base = __ldg(&S->edge_base), es_base = __ldg(&S->es_base);
    const int e0 = edge_base + p0 + f;
    const int kind = __ldg(&S->kind);
    const float sgn = kind == PGM_LOGIC_AND ? -1.f : 1.f;
    if (kind == PGM_LOGIC_XOR)  // uniform over the block (one group per block)
        logic_warp_factor<MAXP, true>(G, b, ev, m_old, m_new, T, damping, e0, n, edge_base, es_base, sgn, sx, spa,
                                      spb, lane);
    else
        logic_warp_factor<MAXP, false>(G, b, ev, m_old, m_new, T, damping, e0, n, edge_base, es_base, sgn, sx, spa,
                                       spb, lane);
}

// =====================================================================================
// Adjoint (gradient of L = sum g * normalised log-beliefs w.r.t. log-potentials and
// evidence, T > 0, enumeration factors). Reverse of each forward step of an iteration:
// the two max-normalisations (the adjoint's sum moves to the argmax state), damping
// (delta to the previous messages, 1 - delta to the factor output), the factor's
// log-sum-exp (a softmax over its configurations), the variable-side sums. In exact
// arithmetic message adjoints sum to zero over each edge's states, but the projection
// of the normalisations must still be applied: rounding seeds a constant component
// that the reverse factor map would otherwise amplify.
// =====================================================================================

// Belief read-out: db = g - softmax(b) * sum(g); d_evidence = db; adjoint of every
// incoming message = db of its variable. Thread per variable.
__global__ void __launch_bounds__(128) k_adj_beliefs(DevGraph G, const float *__restrict__ ev,
                                                     const float *__restrict__ m, const float *__restrict__ gnb,
                                                     float *__restrict__ d_ev, float *__restrict__ adj) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.V) return;
    const int vs = G.vs_off[v], K = G.vs_off[v + 1] - vs, k0 = G.vin_off[v], k1 = G.vin_off[v + 1];
    FF best = ff_make(kNegInf);
    int arg = 0;
    float sg = 0.f;
    for (int x = 0; x < K; ++x) {
        FF s = ff_make(ev[vs + x]);
        for (int k = k0; k < k1; ++k) s = ff_add(s, m[G.vin_es[k] + x]);
        if (x == 0 || ff_gt(s, best)) {
            best = s;
            arg = x;
        }
        sg += gnb[vs + x];
    }
    float z = 0.f;
    for (int x = 0; x < K; ++x) {
        FF s = ff_make(ev[vs + x]);
        for (int k = k0; k < k1; ++k) s = ff_add(s, m[G.vin_es[k] + x]);
        if (x != arg) z += expf(ff_diff(s, best));
    }
    const float lz = log1pf(z);
    for (int x = 0; x < K; ++x) {
        FF s = ff_make(ev[vs + x]);
        for (int k = k0; k < k1; ++k) s = ff_add(s, m[G.vin_es[k] + x]);
        const float r = (x == arg) ? 0.f : ff_diff(s, best);
        const float db = gnb[vs + x] - expf(r - lz) * sg;
        d_ev[vs + x] = db;
        for (int k = k0; k < k1; ++k) adj[G.vin_es[k] + x] = db;
    }
}

// k_adj_factor for a dense pairwise table (K x K, configuration c = x K + y) with K a
// compile-time constant, so that every per-state array stays in registers: the same
// steps, in the same order of operations, as the general loop below (whose arrays of
// kMaxStateSum entries, indexed at run time, live in local memory).
template <int K>
__device__ __forceinline__ void adj_pair_factor(const DevGraph &G, const EnumSeg *S, int f, bool valid,
                                                const float *__restrict__ pot, const float *__restrict__ b,
                                                const float *__restrict__ ev, const float *__restrict__ m_old,
                                                const float *__restrict__ adj, float *__restrict__ dv2f,
                                                float *__restrict__ ddamp, float *__restrict__ d_pot,
                                                float *__restrict__ partials, int nc_max, float T, float invT,
                                                float damping) {
    const int es0 = S->es_base + f * 2 * K, es1 = es0 + K;
    const int e0 = S->edge_base + f * 2;
    float mo0[K], mo1[K], v0[K], v1[K];
    load_n<K>(mo0, m_old + es0);
    load_n<K>(mo1, m_old + es1);
    gather_v2f<K>(G, b, ev, m_old, G.edge_vs[e0], es0, mo0, v0);
    gather_v2f<K>(G, b, ev, m_old, G.edge_vs[e0 + 1], es1, mo1, v1);
    const float *phi = pot + S->pot_base + (S->shared ? 0 : (size_t)f * (K * K));
    // forward values: output 0 at x over y, output 1 at y over x (configurations ascending)
    float l0[K], s0[K], l1[K], s1[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        l0[i] = kNegInf;
        s0[i] = 0.f;
        l1[i] = kNegInf;
        s1[i] = 0.f;
    }
    auto acc = [&](float &lm, float &ls, float s) {
        if (s > lm) {
            ls = ls * expf((lm - s) * invT) + 1.f;
            lm = s;
        } else if (s > kNegInf) {
            ls += expf((s - lm) * invT);
        }
    };
#pragma unroll
    for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) {
            const float p = phi[x * K + y];
            acc(l0[x], s0[x], p + v1[y]);
            acc(l1[y], s1[y], p + v0[x]);
        }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (l0[i] != kNegInf) l0[i] += T * logf(s0[i]);
        if (l1[i] != kNegInf) l1[i] += T * logf(s1[i]);
    }
    // reverse of normalise - damp - normalise, per edge (gam overwrites s)
    const float w1 = (damping != 0.f) ? 1.f - damping : 1.f;
    auto reverse_edge = [&](const float (&lm)[K], const float (&mo)[K], int es, float (&gam)[K]) {
        int a1 = 0;
#pragma unroll
        for (int x = 1; x < K; ++x)
            if (lm[x] > lm[a1]) a1 = x;
        float mx = lm[0];
#pragma unroll
        for (int x = 1; x < K; ++x)
            if (x == a1) mx = lm[x];
        int a2 = 0;
        float d2 = 0.f, sa = 0.f, ad[K];
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const float n = (mx == kNegInf) ? 0.f : lm[x] - mx;
            const float d = (damping != 0.f) ? damping * mo[x] + w1 * n : n;
            if (x == 0 || d > d2) {
                d2 = d;
                a2 = x;
            }
            ad[x] = adj[es + x];
            sa += ad[x];
        }
        float sn = 0.f;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            const float dd = ad[x] - (x == a2 ? sa : 0.f);
            if (valid) ddamp[es + x] = damping * dd;
            gam[x] = w1 * dd;
            sn += gam[x];
        }
#pragma unroll
        for (int x = 0; x < K; ++x)
            if (x == a1) gam[x] -= sn;
    };
    float g0[K], g1[K];
    reverse_edge(l0, mo0, es0, g0);
    reverse_edge(l1, mo1, es1, g1);
    // back through the log-sum-exp
    float dv0[K], dv1[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        dv0[i] = 0.f;
        dv1[i] = 0.f;
    }
    float *dphi = d_pot + S->pot_base + (S->shared ? 0 : (size_t)f * (K * K));
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) {
            const int c = x * K + y;
            const float p = phi[c];
            float dc = 0.f;
            const float sa = p + v1[y];  // output 0 at x
            if (sa != kNegInf && l0[x] != kNegInf) {
                const float w = g0[x] * expf((sa - l0[x]) * invT);
                dc += w;
                dv1[y] += w;
            }
            const float sb = p + v0[x];  // output 1 at y
            if (sb != kNegInf && l1[y] != kNegInf) {
                const float w = g1[y] * expf((sb - l1[y]) * invT);
                dc += w;
                dv0[x] += w;
            }
            if (S->shared) {  // uniform over the warp
                float t = valid ? dc : 0.f;
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
                if (lane == 0) partials[(size_t)gwarp * nc_max + c] = t;
            } else if (valid) {
                dphi[c] += dc;
            }
        }
    if (valid) {
#pragma unroll
        for (int x = 0; x < K; ++x) {
            dv2f[es0 + x] = dv0[x];
            dv2f[es1 + x] = dv1[x];
        }
    }
}

// Factor step in reverse, thread per enumeration factor. From the adjoint a of the new
// messages: dd = a - sum(a) [x == argmax d] (second normalisation), the damping term
// delta * dd goes to `ddamp`, dn = (1 - delta) dd, gamma = dn - sum(dn) [x == argmax mt]
// (first normalisation), and with p_i(c) = exp((s_{-i}(c) - mt_i(c_i)) / T):
//   d log_pot(c) += sum_i gamma_i(c_i) p_i(c)
//   dv2f_j(y)     = sum_{i != j} sum_{c: c_j = y} gamma_i(c_i) p_i(c)
// The variable-to-factor values and mt are recomputed as the forward factor pass does.
// A table shared by the group is not summed into d_pot here: each warp adds its factors'
// contributions in a fixed shuffle order and writes one partial per configuration to
// `partials` (warp w of the launch at w * nc_max), which k_adj_pot_reduce adds to d_pot in
// warp order, so the gradient is the same on every run.
__global__ void __launch_bounds__(128)
k_adj_factor(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
             const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
             const float *__restrict__ adj, float *__restrict__ dv2f, float *__restrict__ ddamp,
             float *__restrict__ d_pot, float *__restrict__ partials, int nc_max, float T, float invT,
             float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int f_raw = (blockIdx.x - S->block_begin) * blockDim.x + threadIdx.x;
    // a block lies in one group, so a warp does; idle lanes shadow the group's last
    // factor (a warp's lanes all take part in the partial sums) and write nothing
    const bool valid = f_raw < S->n_fac;
    if (__all_sync(0xffffffffu, !valid)) return;
    const int f = valid ? f_raw : S->n_fac - 1;
    const int a = S->arity, nc = S->n_cfg, ksum = S->es_per_fac;
    if (S->dense) {  // uniform over the block
        if (S->K[0] == 2) {
            adj_pair_factor<2>(G, S, f, valid, pot, b, ev, m_old, adj, dv2f, ddamp, d_pot, partials, nc_max, T, invT,
                               damping);
            return;
        }
        if (S->K[0] == 4) {
            adj_pair_factor<4>(G, S, f, valid, pot, b, ev, m_old, adj, dv2f, ddamp, d_pot, partials, nc_max, T, invT,
                               damping);
            return;
        }
    }
    int Kj[kMaxArity], Ko[kMaxArity];
    for (int j = 0; j < a; ++j) {
        Kj[j] = S->K[j];
        Ko[j] = S->Koff[j];
    }
    const int es_f = S->es_base + f * ksum;
    const int e_f = S->edge_base + f * a;
    float v2f[kMaxStateSum], gam[kMaxStateSum], lm[kMaxStateSum], ls[kMaxStateSum], dv[kMaxStateSum];
    for (int j = 0; j < a; ++j) {
        const int vs = G.edge_vs[e_f + j];
        const int es = es_f + Ko[j];
        bool exact = false;
        for (int x = 0; x < Kj[j]; ++x) exact |= needs_exact(m_old[es + x]);
        if (vs < 0) {
            float2 hmx = make_float2(-CUDART_INF_F, 0.f);
            for (int x = 0; x < Kj[j]; ++x) {
                const float2 q = hd_pair(G, vs, x, m_old[es + x]);
                if (x == 0 || hd_gt(q, hmx)) hmx = q;
            }
            for (int x = 0; x < Kj[j]; ++x)
                v2f[Ko[j] + x] =
                    hmx.x == -CUDART_INF_F ? -CUDART_INF_F : hd_rel(hd_pair(G, vs, x, m_old[es + x]), hmx);
        } else if (exact) {
            v2f_slow_edge(G, ev, m_old, vs, es, Kj[j], v2f + Ko[j]);
        } else {
            for (int x = 0; x < Kj[j]; ++x) v2f[Ko[j] + x] = b[vs + x] - m_old[es + x];
        }
    }
    for (int i = 0; i < ksum; ++i) {
        lm[i] = kNegInf;
        ls[i] = 0.f;
        dv[i] = 0.f;
    }
    const uint8_t *cfg = G.cfg_pool + S->cfg_base;
    const float *phi = pot + S->pot_base + (S->shared ? 0 : (size_t)f * nc);
    // mt: LSE_T over the configurations consistent with each (edge, state)
    for (int c = 0; c < nc; ++c) {
        const uint8_t *cc = cfg + c * a;
        for (int i = 0; i < a; ++i) {
            float s = phi[c];
            for (int j = 0; j < a; ++j)
                if (j != i) s += v2f[Ko[j] + cc[j]];
            const int idx = Ko[i] + cc[i];
            if (s > lm[idx]) {
                ls[idx] = ls[idx] * expf((lm[idx] - s) * invT) + 1.f;
                lm[idx] = s;
            } else if (s > kNegInf) {
                ls[idx] += expf((s - lm[idx]) * invT);
            }
        }
    }
    for (int i = 0; i < ksum; ++i)
        if (lm[i] != kNegInf) lm[i] += T * logf(ls[i]);
    // reverse of normalise - damp - normalise, per edge
    const float w1 = (damping != 0.f) ? 1.f - damping : 1.f;
    for (int j = 0; j < a; ++j) {
        const int K = Kj[j], o = Ko[j], es = es_f + o;
        int a1 = 0;
        for (int x = 1; x < K; ++x)
            if (lm[o + x] > lm[o + a1]) a1 = x;
        const float mx = lm[o + a1];
        int a2 = 0;
        float d2 = 0.f, sa = 0.f;
        for (int x = 0; x < K; ++x) {
            const float n = (mx == kNegInf) ? 0.f : lm[o + x] - mx;
            const float d = (damping != 0.f) ? damping * m_old[es + x] + w1 * n : n;
            if (x == 0 || d > d2) {
                d2 = d;
                a2 = x;
            }
            sa += adj[es + x];
        }
        float sn = 0.f;
        for (int x = 0; x < K; ++x) {
            const float dd = adj[es + x] - (x == a2 ? sa : 0.f);
            if (valid) ddamp[es + x] = damping * dd;
            gam[o + x] = w1 * dd;
            sn += gam[o + x];
        }
        gam[o + a1] -= sn;
    }
    float *dphi = d_pot + S->pot_base + (S->shared ? 0 : (size_t)f * nc);
    const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    for (int c = 0; c < nc; ++c) {
        const uint8_t *cc = cfg + c * a;
        float dc = 0.f;
        for (int i = 0; i < a; ++i) {
            float s = phi[c];
            for (int j = 0; j < a; ++j)
                if (j != i) s += v2f[Ko[j] + cc[j]];
            const int idx = Ko[i] + cc[i];
            if (s == kNegInf || lm[idx] == kNegInf) continue;
            const float w = gam[idx] * expf((s - lm[idx]) * invT);
            dc += w;
            for (int j = 0; j < a; ++j)
                if (j != i) dv[Ko[j] + cc[j]] += w;
        }
        if (S->shared) {  // uniform over the warp
            float t = valid ? dc : 0.f;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
            if (lane == 0) partials[(size_t)gwarp * nc_max + c] = t;
        } else if (valid) {
            dphi[c] += dc;
        }
    }
    if (valid)
        for (int i = 0; i < ksum; ++i) dv2f[es_f + i] = dv[i];
}

// Adds the warp partials of k_adj_factor to the log-potential gradients of the tables
// shared by a group: block = group record, thread = configuration, warps in ascending
// order (the launch's warp w covers threads 32 w .. 32 w + 31 of its block range).
__global__ void __launch_bounds__(256) k_adj_pot_reduce(const EnumSeg *__restrict__ segs, int n_seg,
                                                        const float *__restrict__ partials, int nc_max,
                                                        int threads_per_block, float *__restrict__ d_pot) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const EnumSeg *S = segs + blockIdx.x;
    if (!S->shared || S->n_fac == 0) return;
    // the group's factors are consecutive from its first block, 32 to a warp; warps past
    // its last factor wrote nothing
    const int w0 = S->block_begin * (threads_per_block >> 5), w1 = w0 + (S->n_fac + 31) / 32;
    for (int c = threadIdx.x; c < S->n_cfg; c += blockDim.x) {
        float sum = 0.f;
        for (int w = w0; w < w1; ++w) sum += partials[(size_t)w * nc_max + c];
        d_pot[S->pot_base + c] += sum;
    }
}

// k_adj_factor for listed-configuration groups with a state sum above kMaxStateSum, with
// the team layout of k_enum_block (a warp per factor up to kEnumWarpStateSum, else the
// block; fpb factors per block; configuration tables read in place). Per factor: the
// variable-to-factor values (enum_team_v2f); each output's forward value lm = LSE_T over
// its configurations (ascending, as k_adj_factor); a warp per edge reverses
// normalise - damp - normalise into gam and ddamp; then gathers in a fixed order: each
// output state walks its configurations and sums the other edges' weights into its
// variable-to-factor adjoint, and each configuration sums its edges' weights into the
// log-potential gradient -- the factor's own table directly, a shared table into the
// team's row of `partials` (team w of block b at (8 b + w) nc_max), which
// k_adj_block_reduce adds to d_pot in order. So the gradient is the same on every run
// (with `partials` null, shared tables fall back to atomic adds).
__global__ void __launch_bounds__(kEnumBlockThreads)
k_adj_block(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
            const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
            const float *__restrict__ adj, float *__restrict__ dv2f, float *__restrict__ ddamp,
            float *__restrict__ d_pot, float *__restrict__ partials, int nc_max, float T, float invT,
            float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    extern __shared__ __align__(16) float ab_smem[];
    __shared__ int sK[kMaxArity], sKo[kMaxArity];
    __shared__ int s_fix[kEnumBlockThreads / 32][kMaxArity];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int a = __ldg(&S->arity), nc = __ldg(&S->n_cfg), ksum = __ldg(&S->es_per_fac);
    const int fpb = __ldg(&S->fpb), n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared);
    const int packed = __ldg(&S->packed);
    const int f0 = (blockIdx.x - __ldg(&S->block_begin)) * fpb;
    const int f1 = min(n_fac, f0 + fpb);
    if (threadIdx.x < a) {
        sK[threadIdx.x] = __ldg(&S->K[threadIdx.x]);
        sKo[threadIdx.x] = __ldg(&S->Koff[threadIdx.x]);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const bool wteam = ksum <= kEnumWarpStateSum;
    const int tsize = wteam ? 32 : (int)blockDim.x, trank = wteam ? lane : (int)threadIdx.x;
    const int team = wteam ? warp : 0, n_teams = wteam ? nw : 1;
    const int ej0 = wteam ? 0 : warp, ejs = wteam ? 1 : nw;
    float *v2f = ab_smem + (size_t)team * 4 * ksum, *lm = v2f + ksum, *gam = lm + ksum, *dv = gam + ksum;
    const uint8_t *cfg = G.cfg_pool + __ldg(&S->cfg_base);
    const int32_t *bs = G.bs_pool + __ldg(&S->bs_base);
    const int32_t *lst = bs + ((ksum + 1 + 3) & ~3);
    const float w1 = (damping != 0.f) ? 1.f - damping : 1.f;
    for (int f = f0 + team; f < f1; f += n_teams) {
        const int es_f = __ldg(&S->es_base) + f * ksum;
        const int e_f = __ldg(&S->edge_base) + f * a;
        const float *phi = pot + __ldg(&S->pot_base) + (shared ? 0 : (size_t)f * nc);
        float *dphi = d_pot + __ldg(&S->pot_base) + (shared ? 0 : (size_t)f * nc);
        enum_team_v2f(G, b, ev, m_old, e_f, es_f, a, ksum, sK, sKo, v2f, nullptr, s_fix[team], wteam, trank, tsize,
                      ej0, ejs, lane);
        // the value s of configuration c seen from output o = (j, x): phi + the other
        // neighbours' variable-to-factor values (for pairwise lists, entry = c << 11 | offset)
        auto value = [&](int o, int j, int ent, int &c) -> float {
            if (packed) {
                c = ent >> 11;
                return __ldg(phi + c) + v2f[ent & 2047];
            }
            c = ent;
            const uint8_t *cc = cfg + (size_t)c * a;
            float sv = __ldg(phi + c);
            for (int k = 0; k < a; ++k)
                if (k != j) sv += v2f[sKo[k] + __ldg(cc + k)];
            return sv;
        };
        // (2) forward values of the outputs
        for (int o = trank; o < ksum; o += tsize) {
            int j = 0;
            for (int k = 1; k < a; ++k)
                if (o >= sKo[k]) j = k;
            float mx = kNegInf, sm = 0.f;
            for (int i = __ldg(bs + o); i < __ldg(bs + o + 1); ++i) {
                int c;
                const float sv = value(o, j, __ldg(lst + i), c);
                if (sv > mx) {
                    sm = sm * expf((mx - sv) * invT) + 1.f;
                    mx = sv;
                } else if (sv > kNegInf) {
                    sm += expf((sv - mx) * invT);
                }
            }
            lm[o] = mx == kNegInf ? mx : mx + T * logf(sm);
            dv[o] = 0.f;
        }
        team_barrier(wteam);
        // (3) reverse of normalise - damp - normalise, a warp per edge
        for (int j = ej0; j < a; j += ejs) {
            const int K = sK[j], o = sKo[j], es = es_f + o;
            float b1 = kNegInf;  // first argmax of lm over the edge
            int a1 = K;
            for (int x = lane; x < K; x += 32)
                if (a1 == K || lm[o + x] > b1) {
                    b1 = lm[o + x];
                    a1 = x;
                }
            for (int d = 16; d > 0; d >>= 1) {
                const float qb = __shfl_xor_sync(0xffffffffu, b1, d);
                const int qa = __shfl_xor_sync(0xffffffffu, a1, d);
                if (qa < K && (a1 == K || qb > b1 || (!(b1 > qb) && qa < a1))) {
                    b1 = qb;
                    a1 = qa;
                }
            }
            const float mx = b1;
            float b2 = kNegInf, sa = 0.f;  // first argmax of the damped value; sum of adj
            int a2 = K;
            for (int x = lane; x < K; x += 32) {
                const float n = (mx == kNegInf) ? 0.f : lm[o + x] - mx;
                const float dd = (damping != 0.f) ? damping * __ldg(m_old + es + x) + w1 * n : n;
                if (a2 == K || dd > b2) {
                    b2 = dd;
                    a2 = x;
                }
                sa += __ldg(adj + es + x);
            }
            for (int d = 16; d > 0; d >>= 1) {
                const float qb = __shfl_xor_sync(0xffffffffu, b2, d);
                const int qa = __shfl_xor_sync(0xffffffffu, a2, d);
                if (qa < K && (a2 == K || qb > b2 || (!(b2 > qb) && qa < a2))) {
                    b2 = qb;
                    a2 = qa;
                }
                sa += __shfl_xor_sync(0xffffffffu, sa, d);
            }
            float sn = 0.f;
            for (int x = lane; x < K; x += 32) {
                const float dd = __ldg(adj + es + x) - (x == a2 ? sa : 0.f);
                ddamp[es + x] = damping * dd;
                gam[o + x] = w1 * dd;
                sn += gam[o + x];
            }
            for (int d = 16; d > 0; d >>= 1) sn += __shfl_xor_sync(0xffffffffu, sn, d);
            __syncwarp();
            if (lane == 0) gam[o + a1] -= sn;
        }
        team_barrier(wteam);
        // (4) back through the log-sum-exp, as gathers in a fixed order (no atomics): the
        // weight of configuration c seen from output o = (j, c_j) is
        // w_j(c) = gam[o] e^((s_j(c) - lm[o]) / T). (4a) The variable-to-factor adjoint of
        // state t of edge k sums w_j(c) over the configurations with c_k = t -- the list of
        // output t -- and the other edges j.
        auto weight = [&](int oj, float sv) -> float {
            if (lm[oj] == kNegInf || sv == kNegInf) return 0.f;
            return gam[oj] * expf((sv - lm[oj]) * invT);
        };
        for (int o = trank; o < ksum; o += tsize) {
            int k = 0;
            for (int q = 1; q < a; ++q)
                if (o >= sKo[q]) k = q;
            float acc = 0.f;
            for (int i = __ldg(bs + o); i < __ldg(bs + o + 1); ++i) {
                const int ent = __ldg(lst + i);
                if (packed) {  // the other edge's output: its state offset is in the entry
                    const int oj = ent & 2047;
                    acc += weight(oj, __ldg(phi + (ent >> 11)) + v2f[o]);
                } else {
                    const uint8_t *cc = cfg + (size_t)ent * a;
                    for (int j = 0; j < a; ++j) {
                        if (j == k) continue;
                        const int oj = sKo[j] + __ldg(cc + j);
                        int c;
                        acc += weight(oj, value(oj, j, ent, c));
                    }
                }
            }
            dv[o] = acc;
        }
        // (4b) the log-potential gradient of configuration c sums w_j(c) over the edges j
        const bool own = partials == nullptr || !shared;
        float *prow = own ? nullptr : partials + ((size_t)blockIdx.x * (kEnumBlockThreads / 32) + team) * nc_max;
        const bool first = (f == f0 + team);  // this team's first factor of the launch
        for (int c = trank; c < nc; c += tsize) {
            const uint8_t *cc = cfg + (size_t)c * a;
            float dc = 0.f;
            for (int j = 0; j < a; ++j) {
                const int oj = sKo[j] + __ldg(cc + j);
                int cx;
                dc += weight(oj, value(oj, j, packed ? ((c << 11) | (sKo[1 - j] + __ldg(cc + 1 - j))) : c, cx));
            }
            if (own) {
                if (partials == nullptr && shared) atomicAdd(dphi + c, dc);  // no scratch: atomics
                else dphi[c] += dc;  // the factor's own table, only this lane writes c
            } else {
                prow[c] = first ? dc : prow[c] + dc;  // the team's row, added over its factors in order
            }
        }
        team_barrier(wteam);
        for (int t = trank; t < ksum; t += tsize) dv2f[es_f + t] = dv[t];
        team_barrier(wteam);  // v2f / lm / dv are reused by the team's next factor
    }
}

// Adds k_adj_block's team rows of the log-potential gradients of shared tables to d_pot:
// block = group record, thread = configuration; the group's blocks in order, and in each
// block the teams that had a factor, in order.
__global__ void __launch_bounds__(256) k_adj_block_reduce(const EnumSeg *__restrict__ segs, int n_seg,
                                                          const float *__restrict__ partials, int nc_max,
                                                          float *__restrict__ d_pot) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const EnumSeg *S = segs + blockIdx.x;
    if (!S->shared || S->n_fac == 0) return;
    const int teams = S->es_per_fac <= kEnumWarpStateSum ? kEnumBlockThreads / 32 : 1;
    const int n_blk = (S->n_fac + S->fpb - 1) / S->fpb;
    for (int c = threadIdx.x; c < S->n_cfg; c += blockDim.x) {
        float sum = 0.f;
        for (int bl = 0; bl < n_blk; ++bl) {
            const int nf = min(S->fpb, S->n_fac - bl * S->fpb);  // factors of this block
            for (int t = 0; t < min(teams, nf); ++t)
                sum += partials[((size_t)(S->block_begin + bl) * (kEnumBlockThreads / 32) + t) * nc_max + c];
        }
        d_pot[S->pot_base + c] += sum;
    }
}

// Reverse of write_logic_edge (t = [-o, 0] or [0, o], then normalise - damp - normalise)
// for one binary edge: mo the old message, ad the adjoint of the new one; writes the
// damping term to ddamp_es[2] and returns the adjoint of o.
__device__ __forceinline__ double logic_edge_reverse(float o, float2 mo, float2 ad, float damping, float *ddamp_es) {
    const float t0 = o >= 0.f ? -o : 0.f, t1 = o >= 0.f ? 0.f : o;
    const int a1 = (t1 > t0) ? 1 : 0;  // first argmax
    const float tm = a1 ? t1 : t0;
    const float w1 = (damping != 0.f) ? 1.f - damping : 1.f;
    const float d0 = (damping != 0.f) ? damping * mo.x + w1 * (t0 - tm) : t0 - tm;
    const float d1 = (damping != 0.f) ? damping * mo.y + w1 * (t1 - tm) : t1 - tm;
    const int a2 = (d1 > d0) ? 1 : 0;
    const float sa = ad.x + ad.y;
    const float dd0 = ad.x - (a2 == 0 ? sa : 0.f), dd1 = ad.y - (a2 == 1 ? sa : 0.f);
    ddamp_es[0] = damping * dd0;
    ddamp_es[1] = damping * dd1;
    float g0 = w1 * dd0, g1 = w1 * dd1;
    const float sn = g0 + g1;
    if (a1 == 0) g0 -= sn;
    else g1 -= sn;
    return o >= 0.f ? -(double)g0 : (double)g1;
}

// Adjoint of the logical OR / AND update (T > 0), thread per factor, in the OR frame
// (AND: inputs and outputs negated). With s_j = sp_T(x_j), A = sum_j s_j, A_-i = A - s_i,
// q = A_-i / T, D_i = log(expm1(q) + e^(-x_c / T)) and cotangents g_i (to parent i) and
// g_c (to the child) on the outgoing log-odds:
//   d out_i / d x_c = e^(-x_c / T - D_i),
//   d out_i / d A_-i = 1 - e^(q - D_i) = expm1(-x_c / T) e^(-D_i),
//   d out_c / d A = L'(A) = e^(A / T) / expm1(A / T),   d s_j / d x_j = sigmoid(x_j / T),
// so dx_c = sum_i g_i e^(-x_c/T - D_i) and dx_j = sigmoid(x_j / T) (g_c L'(A) + H - h_j),
// h_i = g_i d out_i / d A_-i, H = sum_i h_i: linear in the fan-in. The damping term of
// every edge is written as for enumeration factors; a factor with an infinite log-odds
// passes no gradient to its variable-to-factor values.
__global__ void __launch_bounds__(128)
k_adj_logic(DevGraph G, const LogicSeg *__restrict__ segs, int n_seg, const float *__restrict__ b,
            const float *__restrict__ ev, const float *__restrict__ m_old, const float *__restrict__ adj,
            float *__restrict__ dv2f, float *__restrict__ ddamp, float T, float damping) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const LogicSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= __ldg(&S->n_fac)) return;
    const int *po = G.paroff_pool + __ldg(&S->paroff_base);
    const int p0 = __ldg(po + f), n = __ldg(po + f + 1) - p0;
    const int edge_base = __ldg(&S->edge_base), es_base = __ldg(&S->es_base);
    const int e0 = edge_base + p0 + f;
    auto es_of = [&](int k) { return es_base + 2 * (e0 + k - edge_base); };
    const float sgn = __ldg(&S->kind) == 1 ? -1.f : 1.f;
    const double Td = T, invT = 1.0 / Td;
    auto t_of = [&](float x) { return x == kNegInf ? -CUDART_INF : log_softplus_d((double)x * invT); };
    auto adj2 = [&](int es) { return make_float2(__ldg(adj + es), __ldg(adj + es + 1)); };
    // pass 0: child log-odds, log of A / T
    float2 moc;
    const float xc = edge_logodds(G, ev, b, m_old, e0 + n, es_of(n), sgn, moc);
    bool finite = isfinite(xc);
    double la = -CUDART_INF;
    for (int k = 0; k < n; ++k) {
        float2 mo;
        const float x = edge_logodds(G, ev, b, m_old, e0 + k, es_of(k), sgn, mo);
        finite &= isfinite(x);
        la = lse2_d(la, t_of(x));
    }
    const double lm1 = log_expm1_from_log_d(la);
    // the child edge
    const double gc = sgn * logic_edge_reverse(sgn * (float)(Td * lm1), moc, adj2(es_of(n)), damping,
                                               ddamp + es_of(n));
    finite &= n > 0 && la != -CUDART_INF;
    const double lc = -(double)xc * invT;
    // pass 1: each parent's output and damping term; dx_c; h_i (kept in FP64 in the
    // parent's two dv2f words meanwhile). h_i grows like 1 / q when the other parents are
    // off, so the largest h is kept apart (hm, index km) from the sum of the others (Hx),
    // and H - h_j never subtracts it.
    double dxc = 0.0, Hx = 0.0, hm = 0.0;
    int km = -1;
    for (int i = 0; i < n; ++i) {
        float2 mo;
        const float xi = edge_logodds(G, ev, b, m_old, e0 + i, es_of(i), sgn, mo);
        const double ti = t_of(xi);
        double li;  // log(A_-i / T)
        if (ti == -CUDART_INF) {
            li = la;
        } else if (ti - la < -0.7) {
            li = la + log(-expm1(ti - la));
        } else {  // parent i carries most of A: the explicit leave-one-out sum
            li = -CUDART_INF;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                float2 mj;
                li = lse2_d(li, t_of(edge_logodds(G, ev, b, m_old, e0 + j, es_of(j), sgn, mj)));
            }
        }
        const double gi = sgn * logic_edge_reverse(sgn * or_parent_soft(li, xc, Td), mo, adj2(es_of(i)), damping,
                                                   ddamp + es_of(i));
        double hi = 0.0;
        if (finite) {
            const double D = lse2_d(log_expm1_from_log_d(li), lc);
            dxc += gi * exp(lc - D);
            hi = gi * expm1(lc) * exp(-D);
            if (km < 0 || fabs(hi) > fabs(hm)) {
                if (km >= 0) Hx += hm;
                hm = hi;
                km = i;
            } else {
                Hx += hi;
            }
        }
        reinterpret_cast<double *>(dv2f + es_of(i))[0] = hi;  // (es_of is even: 8-byte aligned)
    }
    if (!finite) {
        for (int k = 0; k <= n; ++k) {
            dv2f[es_of(k)] = 0.f;
            dv2f[es_of(k) + 1] = 0.f;
        }
        return;
    }
    // pass 2: the parents' adjoints, then the child's (x = sgn (a1 - a0))
    const double cA = gc * exp(exp(la) - lm1);  // g_c L'(A)
    for (int j = 0; j < n; ++j) {
        float2 mo;
        const float xj = edge_logodds(G, ev, b, m_old, e0 + j, es_of(j), sgn, mo);
        const double sj = 1.0 / (1.0 + exp(-(double)xj * invT));
        const double hj = reinterpret_cast<const double *>(dv2f + es_of(j))[0];
        const double Hj = (j == km) ? Hx : hm + (Hx - hj);  // H - h_j
        const double dxj = sj * (cA + Hj);
        dv2f[es_of(j)] = (float)(-sgn * dxj);
        dv2f[es_of(j) + 1] = (float)(sgn * dxj);
    }
    dv2f[es_of(n)] = (float)(-sgn * dxc);
    dv2f[es_of(n) + 1] = (float)(sgn * dxc);
}

// Variable step in reverse for binary graphs with the padded 4-edge table (vin_tab4):
// the same sums in the same order as k_adj_var below, both states at once (8-byte loads
// and stores, one table row instead of the CSR offsets and list), so the same bits.
__global__ void __launch_bounds__(64) k_adj_var_tab4(DevGraph G, const float *__restrict__ ddamp,
                                                     const float *__restrict__ dv2f, float *__restrict__ adj_prev,
                                                     float *__restrict__ d_ev) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.V) return;
    const int4 t = __ldg(G.vin_tab4 + v);
    const int es[4] = {t.x, t.y, t.z, t.w};
    float2 q[4];
    FF d0 = ff_make(0.f), d1 = ff_make(0.f);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (es[k] >= 0) {
            q[k] = *reinterpret_cast<const float2 *>(dv2f + es[k]);
            d0 = ff_add(d0, q[k].x);
            d1 = ff_add(d1, q[k].y);
        }
    const float a0 = d0.hi + d0.lo, a1 = d1.hi + d1.lo;
    float2 *de = reinterpret_cast<float2 *>(d_ev) + v;  // binary: states at 2v
    float2 e = *de;
    e.x += a0;
    e.y += a1;
    *de = e;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (es[k] >= 0) {
            const float2 dd = *reinterpret_cast<const float2 *>(ddamp + es[k]);
            *reinterpret_cast<float2 *>(adj_prev + es[k]) = make_float2(dd.x - q[k].x + a0, dd.y - q[k].y + a1);
        }
}

// Variable step in reverse, thread per variable: db(x) = sum over incoming edges of
// dv2f(x); d_evidence += db; adjoint of message m_{t-1} on each incoming edge =
// ddamp - dv2f + db (ddamp: the damping term from k_adj_factor).
__global__ void __launch_bounds__(128) k_adj_var(DevGraph G, const float *__restrict__ ddamp,
                                                 const float *__restrict__ dv2f, float *__restrict__ adj_prev,
                                                 float *__restrict__ d_ev) {
    pdl_wait();  // inputs of the previous launch
    pdl_launch_dependents();  // the next launch may be scheduled (it waits likewise)
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.V) return;
    const int vs = G.vs_off[v], K = G.vs_off[v + 1] - vs, k0 = G.vin_off[v], k1 = G.vin_off[v + 1];
    for (int x = 0; x < K; ++x) {
        FF db = ff_make(0.f);
        for (int k = k0; k < k1; ++k) db = ff_add(db, dv2f[G.vin_es[k] + x]);
        const float d = db.hi + db.lo;
        d_ev[vs + x] += d;
        for (int k = k0; k < k1; ++k) {
            const int i = G.vin_es[k] + x;
            adj_prev[i] = ddamp[i] - dv2f[i] + d;
        }
    }
}

// =====================================================================================
// Binary pairwise graphs: log-ratio messages (Plan::lr)
// =====================================================================================
//
// After the epilogue (normalise, damp, normalise) a binary message has one entry that is
// exactly 0 and the other <= 0, so d = m(1) - m(0) stores it in one float without loss:
// m = (-d, 0) for d > 0, else (0, d); both directions are exact (a subtraction from 0, a
// negation). Iterations on a graph whose variables are all binary and whose factors are
// all 2 x 2 tables (F factors, E = 2F edges; edge e = 2g + j is slot j of factor g, its
// states at 2e) keep two arrays of S floats in variable order:
//   d    the factor-to-variable messages as log-ratios;
//   lam  the variable-to-factor values as log-ratios, lam = l(1) - l(0) with
//        l(x) = e_v(x) + sum over the variable's other edges of m(x), the leave-one-out
//        sum (no rounded b - m, so no threshold fallback is needed).
// Position of an edge (G.lr_pos[e]): on graphs whose variables have at most 4 factors,
// k V + v for the k-th incoming edge of variable v (S = 4V; the unused slots of d stay
// 0, which adds nothing to a log-ratio sum, and their lam is never read); otherwise the
// edge's index in the variables' CSR order (S = E). The variable pass streams d and
// lam in variable order with no index (four coalesced streams on the 4-slot layout); the
// factor pass streams lr_pos and the potentials in factor order and gathers / scatters
// lam and d (L2-resident between the passes), updating d in place (an edge's slot
// belongs to one factor). A leave-one-out pair that is -inf in both states
// (contradictory evidence) is stored as the NaN pattern kLamBothNegInf; FP32 arithmetic
// on this GPU returns the canonical NaN 0x7fffffff, never this pattern.

constexpr uint32_t kLamBothNegInf = 0x7fc00001u;

// Programmatic dependent launch between the passes of a log-ratio run (the kernels are
// launched with cudaLaunchAttributeProgrammaticStreamSerialization): each pass lets the
// next one be scheduled as soon as all of its own blocks have started, loads only inputs
// that are fixed for the run before pdl_wait(), and reads or writes the arrays the
// passes exchange only after it. pdl_wait() returns once the previous kernel of the
// stream has completed and its writes are visible (at once when there is none); as
// that kernel waited the same way, every earlier one has completed too.

__device__ __forceinline__ float2 lr_decode(float d) {
    return d > 0.f ? make_float2(-d, 0.f) : make_float2(0.f, d);
}

__device__ __forceinline__ float lr_encode(float m0, float m1) { return m1 - m0; }

__device__ __forceinline__ float2 lam_decode(float l) {
    if (__float_as_uint(l) == kLamBothNegInf) return make_float2(kNegInf, kNegInf);
    return lr_decode(l);
}

__device__ __forceinline__ float lam_encode(FF l0, FF l1) {
    if (l0.hi == kNegInf && l1.hi == kNegInf) return __uint_as_float(kLamBothNegInf);
    return ff_diff(l1, l0);
}

// ff_add for operands known to be finite: an overflow shows as a non-finite result,
// which the caller tests.
__device__ __forceinline__ FF ff_add_nc(FF a, float v) {
    const float s = a.hi + v;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (v - bp);
    return FF{s, a.lo + e};
}

// Variable-to-factor log-ratios of one variable: the leave-one-out value of edge k is
//   lam_k = l_k(1) - l_k(0) = (e(1) - e(0)) + sum over j != k of d_j = D - d_k,
// linear in the stored log-ratios, with D = (e(1) - e(0)) + sum_j d_j kept float-float
// (the evidence difference exactly, by TwoSum), so lam_k is exact up to its final
// rounding. lr_var_slow handles a variable with an infinite evidence entry or message
// (hard constraints) by the per-state explicit sums l_k(x) instead (d = 0 of an unused
// slot decodes to (0, 0) and adds nothing there either).
__device__ __noinline__ void lr_var_slow(float2 e, const float *dk, const int *pos, int n, float *lam) {
    for (int k = 0; k < n; ++k) {
        FF l0 = ff_make(e.x), l1 = ff_make(e.y);
        for (int j = 0; j < n; ++j) {
            if (j == k) continue;
            const float2 q = lr_decode(dk[j]);
            l0 = ff_add(l0, q.x);
            l1 = ff_add(l1, q.y);
        }
        lam[pos[k]] = lam_encode(l0, l1);
    }
}

// Variable pass, at most 4 factors per variable: thread per variable, slot k of variable
// v at k V + v; four coalesced loads of d and one store per variable, no index. It
// writes the float-float total D = (e(1) - e(0)) + sum_k d_k (Dv[v] = (hi, lo)); the
// factor pass forms each edge's lam = D - d_k itself, with the same arithmetic (it
// reads d_k for the damping anyway), which halves the bytes this pass writes. A
// variable whose lam would not come out finite this way (an infinite evidence entry or
// message; an overflow) gets its four lam by the per-state explicit sums in lam, and
// the pattern kDvSlow in Dv[v].x so that the factor pass reads them there.
constexpr uint32_t kDvSlow = 0x7fc00002u;

__device__ __forceinline__ float lr_lam_from_D(float2 D, float dk) {
    const FF l = ff_add_nc(FF{D.x, D.y}, -dk);
    return l.hi + l.lo;
}

__global__ void __launch_bounds__(256) k_var_slot4_lr(int V, const float *__restrict__ ev,
                                                      const float *__restrict__ d, float2 *__restrict__ Dv,
                                                      float *__restrict__ lam) {
    pdl_launch_dependents();
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float2 e = __ldcs(reinterpret_cast<const float2 *>(ev) + v);
    pdl_wait();  // d is the previous factor pass's output
    float dk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dk[k] = __ldcg(d + (size_t)k * V + v);
    bool fin = isfinite(e.x) & isfinite(e.y);
#pragma unroll
    for (int k = 0; k < 4; ++k) fin &= isfinite(dk[k]);
    if (fin) {
        FF D = ff_add_nc(ff_make(e.y), -e.x);
#pragma unroll
        for (int k = 0; k < 4; ++k) D = ff_add_nc(D, dk[k]);
        const float2 Df = make_float2(D.hi, D.lo);
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) ok &= isfinite(lr_lam_from_D(Df, dk[k]));
        if (ok) {
            Dv[v] = Df;
            return;
        }
    }
    // an infinite entry, or an intermediate overflow (inputs near the FP32 range)
    const int pos[4] = {v, V + v, 2 * V + v, 3 * V + v};
    lr_var_slow(e, dk, pos, 4, lam);
    Dv[v] = make_float2(__uint_as_float(kDvSlow), 0.f);
}

// Variable pass, CSR layout (a variable's edges at vin_off[v] .. vin_off[v + 1] - 1, at
// most kVarBlockDegree of them): thread per variable, one pass for D, one for the edges.
__global__ void __launch_bounds__(256) k_var_csr_lr(DevGraph G, const int32_t *__restrict__ list, int n,
                                                    const float *__restrict__ ev, const float *__restrict__ d,
                                                    float *__restrict__ lam) {
    pdl_launch_dependents();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int v = list ? __ldg(list + t) : t;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    const float2 e = __ldg(reinterpret_cast<const float2 *>(ev) + v);  // all binary: states at 2v
    pdl_wait();  // d is the previous factor pass's output
    bool fin = isfinite(e.x) & isfinite(e.y);
    FF D = ff_add(ff_make(e.y), -e.x);
    for (int k = k0; k < k1; ++k) {
        const float dv = __ldcg(d + k);
        fin &= isfinite(dv);
        D = ff_add(D, dv);
    }
    if (fin) {
        for (int k = k0; k < k1; ++k) {
            const FF l = ff_add(D, -__ldcg(d + k));
            lam[k] = l.hi + l.lo;
        }
        return;
    }
    // an infinite entry: per-state explicit sums
    for (int k = k0; k < k1; ++k) {
        FF l0 = ff_make(e.x), l1 = ff_make(e.y);
        for (int j = k0; j < k1; ++j) {
            if (j == k) continue;
            const float2 r = lr_decode(__ldcg(d + j));
            l0 = ff_add(l0, r.x);
            l1 = ff_add(l1, r.y);
        }
        lam[k] = lam_encode(l0, l1);
    }
}

// LSE_T of two values for the log-ratio factor pass:
//   max + T ln(1 + e^((min - max) / T)) = max + (T ln 2) log2(1 + 2^((min - max) k)),
// k = log2(e) / T, on the SFU's base-2 exponential and logarithm (flush-to-zero forms;
// the argument of log2 lies in [1, 2], the result's absolute error is below 3e-7 T).
__device__ __forceinline__ float lse2_fast(float a, float b, float k, float Tln2) {
    const float mx = fmaxf(a, b), mn = fminf(a, b);
    float p, l;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"((mn - mx) * k));
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(1.f + p));
    return fmaf(Tln2, l, mx);
}

// The same with the -inf case (both values -inf) returning -inf.
template <bool MAXP>
__device__ __forceinline__ float lse2_lr(float a, float b, float k, float Tln2) {
    if constexpr (MAXP) return fmaxf(a, b);
    if (fmaxf(a, b) == kNegInf) return kNegInf;
    return lse2_fast(a, b, k, Tln2);
}

template <bool MAXP>
__device__ __forceinline__ float lse2_fast_t(float a, float b, float k, float Tln2) {
    if constexpr (MAXP) return fmaxf(a, b);
    else return lse2_fast(a, b, k, Tln2);
}

// The normalise-damp-normalise epilogue (finish_k) in log-ratio form: from the factor's
// values a(0), a(1) and the stored message d_old, the new message's log-ratio. The
// decoded pairs are those finish_k sees, so the result is the one it would store; a
// contradiction (both entries -inf) gives zeros and the flag.
__device__ __forceinline__ float lr_finish(float a0, float a1, float d_old, float damping, uint32_t *flags) {
    float dt;
    if (a0 == kNegInf && a1 == kNegInf) {
        atomicOr(flags, kFlagContradiction);
        dt = 0.f;
    } else {
        dt = a1 - a0;
    }
    if (damping == 0.f) return dt;
    const float2 o = lr_decode(dt), mo = lr_decode(d_old);
    const float w = 1.f - damping;
    const float t0 = damping * mo.x + w * o.x, t1 = damping * mo.y + w * o.y;
    if (t0 == kNegInf && t1 == kNegInf) {
        atomicOr(flags, kFlagContradiction);
        return 0.f;
    }
    return t1 - t0;
}

// One factor's two new log-ratio messages with every special case handled: a
// variable-to-factor pair that is -inf in both states, table entries of -inf, infinite
// stored messages, damping 0 (the update of finish_k, decoded pair by pair).
template <bool MAXP>
__device__ __noinline__ float2 pair2_lr_exact(const float *phi, float l0, float l1, float mo0, float mo1,
                                              float k, float Tln2, float damping, uint32_t *flags) {
    const float2 v0 = lam_decode(l0), v1 = lam_decode(l1);
    const float a0 = lse2_lr<MAXP>(phi[0] + v1.x, phi[1] + v1.y, k, Tln2);
    const float a1 = lse2_lr<MAXP>(phi[2] + v1.x, phi[3] + v1.y, k, Tln2);
    const float c0 = lse2_lr<MAXP>(phi[0] + v0.x, phi[2] + v0.y, k, Tln2);
    const float c1 = lse2_lr<MAXP>(phi[1] + v0.x, phi[3] + v0.y, k, Tln2);
    return make_float2(lr_finish(a0, a1, mo0, damping, flags), lr_finish(c0, c1, mo1, damping, flags));
}

// The segment of global factor g (segments in factor order, segment i starting at
// factor segs[i].edge_base / 2).
__device__ __forceinline__ int lr_seg_of(const EnumSeg *__restrict__ segs, int n_seg, int g) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((__ldg(&segs[mid].edge_base) >> 1) <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The table of global factor g: its own 4 entries, or the segment's shared table.
__device__ __forceinline__ float4 lr_table(const EnumSeg *__restrict__ segs, int n_seg,
                                           const float *__restrict__ pot, int g) {
    const EnumSeg *S = segs + lr_seg_of(segs, n_seg, g);
    const int shared = __ldg(&S->shared);
    const float *t = pot + __ldg(&S->pot_base) + (shared ? 0 : (size_t)4 * (g - (__ldg(&S->edge_base) >> 1)));
    if ((reinterpret_cast<uintptr_t>(t) & 15u) == 0)
        return shared ? __ldg(reinterpret_cast<const float4 *>(t)) : __ldcs(reinterpret_cast<const float4 *>(t));
    return make_float4(__ldg(t), __ldg(t + 1), __ldg(t + 2), __ldg(t + 3));
}

// Per run: each factor's table as the three numbers the log-ratio update depends on,
// c = phi(1,0) - phi(0,0), al = phi(1,1) - phi(1,0), be = phi(0,1) - phi(0,0), at
// prm[g], prm[F + g], prm[2F + g]. A table with a non-finite entry gets c = NaN, which
// sends its factor to the exact path (that reads the table itself).
__global__ void __launch_bounds__(256) k_lr_params(const EnumSeg *__restrict__ segs, int n_seg, int F,
                                                   const float *__restrict__ pot, float *__restrict__ prm) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= F) return;
    const float4 t = lr_table(segs, n_seg, pot, g);
    const bool fin = isfinite(t.x) & isfinite(t.y) & isfinite(t.z) & isfinite(t.w);
    prm[g] = fin ? t.z - t.x : CUDART_NAN_F;
    prm[F + g] = t.w - t.z;
    prm[2 * (size_t)F + g] = t.y - t.x;
}

// sp_T(x) = T ln(1 + e^(x / T)) = max(x, 0) + (T ln 2) log2(1 + 2^(-|x| k)), k = log2(e) / T,
// on the SFU's base-2 exponential and logarithm (flush-to-zero forms; the argument of
// log2 lies in [1, 2], absolute error below 3e-7 T); max(x, 0) for T = 0.
template <bool MAXP>
__device__ __forceinline__ float softplus_t(float x, float k, float Tln2) {
    if constexpr (MAXP) {
        return fmaxf(x, 0.f);
    } else {
        float p, l;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(p) : "f"(-fabsf(x) * k));
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(1.f + p));
        return fmaf(Tln2, l, fmaxf(x, 0.f));
    }
}

// Factor pass, 2 x 2 tables, persistent: thread-stride loop over the global factors
// g = 0 .. F-1 (edges 2g to its variable 0 and 2g + 1, at slots p = lr_pos[2g],
// lr_pos[2g + 1] of lam and d; FROM_D: the 4-slot layout, lam formed from the
// variable's total Dv and d as in k_var_slot4_lr), software-pipelined: the slots and the
// table numbers of the next factor are loaded before the current factor's gathers and
// arithmetic, so the index stream's latency overlaps the gathers'. d is updated in place
// (a slot belongs to one factor).
//
// With the variable-to-factor log-ratios l0, l1 and the table numbers (k_lr_params),
// LSE_T over the other variable's states gives the new log-ratios
//   to variable 0: c  + sp_T(al + l1) - sp_T(be + l1),
//   to variable 1: be + sp_T(al + c - be + l0) - sp_T(c + l0)   (al + c - be = phi(1,1) - phi(0,1)).
// With o, mo the decoded new and stored messages (one entry of each exactly 0), the damped
// pair t = damping mo + (1 - damping) o has log-ratio damping d_old + (1 - damping) dt,
// since min(x, 0) + max(x, 0) = x; the final normalisation does not change it. Every
// input that needs the guarded arithmetic (a non-finite table entry, an infinite
// variable-to-factor value or stored message, damping 0 against an infinite stored
// message) makes a result non-finite; that and a NaN lam (the contradiction pattern)
// send the factor to pair2_lr_exact with its table.
template <bool MAXP, bool FROM_D>
__global__ void __launch_bounds__(256) k_pair2_lr(const EnumSeg *__restrict__ segs, int n_seg, int F, int V,
                                                  const int2 *__restrict__ lr_pos2, const float *__restrict__ prm,
                                                  const float *__restrict__ pot, const float2 *__restrict__ Dv,
                                                  const float *__restrict__ lam, float *__restrict__ d,
                                                  uint32_t *flags, float k, float Tln2, float damping) {
    pdl_launch_dependents();
    const int stride = gridDim.x * blockDim.x;
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= F) return;
    int2 p = __ldcs(lr_pos2 + g);
    float c = __ldcs(prm + g), al = __ldcs(prm + F + g), be = __ldcs(prm + 2 * (size_t)F + g);
    const float w = 1.f - damping;
    pdl_wait();  // Dv / lam are the variable pass's output
    while (true) {
        const int gn = g + stride;
        int2 pn = p;
        float cn = c, aln = al, ben = be;
        if (gn < F) {
            pn = __ldcs(lr_pos2 + gn);
            cn = __ldcs(prm + gn);
            aln = __ldcs(prm + F + gn);
            ben = __ldcs(prm + 2 * (size_t)F + gn);
        }
        const float mo0 = __ldcg(d + p.x), mo1 = __ldcg(d + p.y);
        float l0, l1;
        if constexpr (FROM_D) {
            // the slots' variables: slot k V + v, k = 0..3
            const int v0 = p.x - V * ((p.x >= V) + (p.x >= 2 * V) + (p.x >= 3 * V));
            const int v1 = p.y - V * ((p.y >= V) + (p.y >= 2 * V) + (p.y >= 3 * V));
            const float2 D0 = __ldcg(Dv + v0), D1 = __ldcg(Dv + v1);
            l0 = __float_as_uint(D0.x) == kDvSlow ? __ldcg(lam + p.x) : lr_lam_from_D(D0, mo0);
            l1 = __float_as_uint(D1.x) == kDvSlow ? __ldcg(lam + p.y) : lr_lam_from_D(D1, mo1);
        } else {
            l0 = __ldcg(lam + p.x);
            l1 = __ldcg(lam + p.y);
        }
        const float dt0 = c + softplus_t<MAXP>(al + l1, k, Tln2) - softplus_t<MAXP>(be + l1, k, Tln2);
        const float dt1 = be + softplus_t<MAXP>(al + c - be + l0, k, Tln2) - softplus_t<MAXP>(c + l0, k, Tln2);
        float2 dn = make_float2(fmaf(damping, mo0, w * dt0), fmaf(damping, mo1, w * dt1));
        if (!(isfinite(dn.x) && isfinite(dn.y) && l0 == l0 && l1 == l1)) {
            const float4 t = lr_table(segs, n_seg, pot, g);
            const float t4[4] = {t.x, t.y, t.z, t.w};
            dn = pair2_lr_exact<MAXP>(t4, l0, l1, mo0, mo1, k, Tln2, damping, flags);
        }
        d[p.x] = dn.x;
        d[p.y] = dn.y;
        if (gn >= F) break;
        g = gn;
        p = pn;
        c = cn;
        al = aln;
        be = ben;
    }
}

// Pack: the log-ratios of msgs ([2E] edge-state layout) into d in variable order (exact
// for max-normalised messages, else the normalised message's log-ratio, to which the
// next update is invariant); unused slots get 0. Unpack: every edge's two entries
// = lr_decode of its slot.
__global__ void __launch_bounds__(256) k_lr_pack_slot4(DevGraph G, const float *__restrict__ m,
                                                       float *__restrict__ d) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= G.V) return;
    const int4 t = __ldg(G.vin_tab4 + v);
    const int es[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
        d[(size_t)k * G.V + v] = es[k] >= 0 ? lr_encode(__ldg(m + es[k]), __ldg(m + es[k] + 1)) : 0.f;
}

__global__ void __launch_bounds__(256) k_lr_pack_csr(DevGraph G, const float *__restrict__ m,
                                                     float *__restrict__ d) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G.E) return;
    const int es = __ldg(G.vin_es + k);
    d[k] = lr_encode(__ldg(m + es), __ldg(m + es + 1));
}

template <bool ALIGNED>
__global__ void __launch_bounds__(256) k_lr_unpack(DevGraph G, const float *__restrict__ d,
                                                   float *__restrict__ m) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= G.E) return;
    const float2 q = lr_decode(__ldg(d + __ldg(G.lr_pos + e)));
    if constexpr (ALIGNED) {
        reinterpret_cast<float2 *>(m)[e] = q;
    } else {
        m[2 * (size_t)e] = q.x;
        m[2 * (size_t)e + 1] = q.y;
    }
}

// =====================================================================================
// Many evidence / potential sets on one binary pairwise graph (pgm_run_bp_multi)
// =====================================================================================
//
// S samples share the graph's structure (4-slot log-ratio layout). The arrays put the
// sample index innermost: slot p of sample s at p S + s, variable v of sample s at
// v S + s, table numbers of factor g at g Sp + s (Sp = S for per-sample tables, else 1
// and shared). Thread (item) t = i S + s works on sample s of variable / factor i, so
// consecutive threads read consecutive samples (coalesced) and the S threads of one
// factor share its slot pair and, with a shared table, its table numbers. The
// per-sample arithmetic is that of the single-sample kernels, step for step.

// Per run: the evidence pairs in variable-major, sample-minor order (ev_s[v S + s]).
__global__ void __launch_bounds__(256) k_ms_evidence(int V, int S, int64_t VS, const float *__restrict__ ev,
                                                     float2 *__restrict__ ev_s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)V * S) return;
    const int v = (int)(t / S), s = (int)(t - (int64_t)v * S);
    const float *e = ev + (size_t)s * VS + 2 * (size_t)v;
    ev_s[t] = make_float2(__ldg(e), __ldg(e + 1));
}

// Per run: the log-ratios of each sample's messages ([S][2E] edge-state layout) into
// slot-major, sample-minor d; unused slots 0 (as k_lr_pack_slot4).
__global__ void __launch_bounds__(256) k_ms_pack(DevGraph G, int S, const float *__restrict__ m,
                                                 float *__restrict__ d) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)G.V * S) return;
    const int v = (int)(t / S), s = (int)(t - (int64_t)v * S);
    const int4 q = __ldg(G.vin_tab4 + v);
    const int es[4] = {q.x, q.y, q.z, q.w};
    const float *ms = m + (size_t)s * G.ES;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        d[((size_t)k * G.V + v) * S + s] = es[k] >= 0 ? lr_encode(__ldg(ms + es[k]), __ldg(ms + es[k] + 1)) : 0.f;
}

// Per run: each sample's messages back into the [S][2E] edge-state layout.
__global__ void __launch_bounds__(256) k_ms_unpack(DevGraph G, int S, const float *__restrict__ d,
                                                   float *__restrict__ m) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)G.E * S) return;
    const int s = (int)(t / G.E), e = (int)(t - (int64_t)s * G.E);
    const float2 q = lr_decode(__ldg(d + (size_t)__ldg(G.lr_pos + e) * S + s));
    float *ms = m + (size_t)s * G.ES + 2 * (size_t)e;
    ms[0] = q.x;
    ms[1] = q.y;
}

// Per run: table differences (k_lr_params) of each of the Sp table sets (pot + sp P),
// at prm[g Sp + sp], prm[F Sp + g Sp + sp], prm[2 F Sp + g Sp + sp].
__global__ void __launch_bounds__(256) k_ms_params(const EnumSeg *__restrict__ segs, int n_seg, int F, int Sp,
                                                   int64_t P, const float *__restrict__ pot,
                                                   float *__restrict__ prm) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)F * Sp;
    if (t >= n) return;
    const int g = (int)(t / Sp), sp = (int)(t - (int64_t)g * Sp);
    const float4 q = lr_table(segs, n_seg, pot + (size_t)sp * P, g);
    const bool fin = isfinite(q.x) & isfinite(q.y) & isfinite(q.z) & isfinite(q.w);
    prm[t] = fin ? q.z - q.x : CUDART_NAN_F;
    prm[n + t] = q.w - q.z;
    prm[2 * n + t] = q.y - q.x;
}

// Variable pass (k_var_slot4_lr per sample): item t = v S + s.
__global__ void __launch_bounds__(256) k_ms_var(int V, int S, const float2 *__restrict__ ev_s,
                                                const float *__restrict__ d, float2 *__restrict__ Dv,
                                                float *__restrict__ lam) {
    pdl_launch_dependents();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)V * S) return;
    const float2 e = __ldcs(ev_s + t);
    const size_t plane = (size_t)V * S;  // one slot index k across all variables and samples
    pdl_wait();  // d is the previous factor pass's output
    float dk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) dk[k] = __ldcg(d + k * plane + t);
    bool fin = isfinite(e.x) & isfinite(e.y);
#pragma unroll
    for (int k = 0; k < 4; ++k) fin &= isfinite(dk[k]);
    if (fin) {
        FF D = ff_add_nc(ff_make(e.y), -e.x);
#pragma unroll
        for (int k = 0; k < 4; ++k) D = ff_add_nc(D, dk[k]);
        const float2 Df = make_float2(D.hi, D.lo);
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) ok &= isfinite(lr_lam_from_D(Df, dk[k]));
        if (ok) {
            Dv[t] = Df;
            return;
        }
    }
    const int pos[4] = {(int)t, (int)(plane + t), (int)(2 * plane + t), (int)(3 * plane + t)};
    lr_var_slow(e, dk, pos, 4, lam);
    Dv[t] = make_float2(__uint_as_float(kDvSlow), 0.f);
}

// Factor pass (k_pair2_lr<MAXP, FROM_D> per sample): item t = g S + s, grid-stride.
// The S items of factor g read its slot pair (one 8-byte load, the same address) and,
// with Sp = 1, its table numbers; lam / d / Dv are gathered per sample at p S + s and
// v S + s.
template <bool MAXP>
__global__ void __launch_bounds__(256) k_ms_pair(const EnumSeg *__restrict__ segs, int n_seg, int F, int V, int S,
                                                 int Sp, int64_t P, const int2 *__restrict__ lr_pos2,
                                                 const float *__restrict__ prm, const float *__restrict__ pot,
                                                 const float2 *__restrict__ Dv, const float *__restrict__ lam,
                                                 float *__restrict__ d, uint32_t *flags, float k, float Tln2,
                                                 float damping) {
    pdl_launch_dependents();
    const int64_t n = (int64_t)F * S, np = (int64_t)F * Sp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float w = 1.f - damping;
    bool waited = false;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
        const int g = (int)(t / S), s = (int)(t - (int64_t)g * S);
        const int2 p = __ldg(lr_pos2 + g);
        const int64_t q = (int64_t)g * Sp + (Sp > 1 ? s : 0);
        const float c = __ldg(prm + q), al = __ldg(prm + np + q), be = __ldg(prm + 2 * np + q);
        if (!waited) {
            pdl_wait();  // Dv / lam are the variable pass's output
            waited = true;
        }
        const size_t px = (size_t)p.x * S + s, py = (size_t)p.y * S + s;
        const float mo0 = __ldcg(d + px), mo1 = __ldcg(d + py);
        const int v0 = p.x - V * ((p.x >= V) + (p.x >= 2 * V) + (p.x >= 3 * V));
        const int v1 = p.y - V * ((p.y >= V) + (p.y >= 2 * V) + (p.y >= 3 * V));
        const float2 D0 = __ldcg(Dv + (size_t)v0 * S + s), D1 = __ldcg(Dv + (size_t)v1 * S + s);
        const float l0 = __float_as_uint(D0.x) == kDvSlow ? __ldcg(lam + px) : lr_lam_from_D(D0, mo0);
        const float l1 = __float_as_uint(D1.x) == kDvSlow ? __ldcg(lam + py) : lr_lam_from_D(D1, mo1);
        const float dt0 = c + softplus_t<MAXP>(al + l1, k, Tln2) - softplus_t<MAXP>(be + l1, k, Tln2);
        const float dt1 = be + softplus_t<MAXP>(al + c - be + l0, k, Tln2) - softplus_t<MAXP>(c + l0, k, Tln2);
        float2 dn = make_float2(fmaf(damping, mo0, w * dt0), fmaf(damping, mo1, w * dt1));
        if (!(isfinite(dn.x) && isfinite(dn.y) && l0 == l0 && l1 == l1)) {
            const float4 tq = lr_table(segs, n_seg, pot + (Sp > 1 ? (size_t)s * P : 0), g);
            const float t4[4] = {tq.x, tq.y, tq.z, tq.w};
            dn = pair2_lr_exact<MAXP>(t4, l0, l1, mo0, mo1, k, Tln2, damping, flags);
        }
        d[px] = dn.x;
        d[py] = dn.y;
    }
}

// Perturb-and-max-product: sample s's evidence = evidence + noise[s] (all samples).
__global__ void __launch_bounds__(256) k_pmp_perturb(int64_t VS, int S, const float *__restrict__ ev,
                                                     const float *__restrict__ noise, float *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= VS * S) return;
    out[t] = __ldg(ev + t % VS) + __ldg(noise + t);
}

// Residual of one iteration: *out = max over i of |a[i] - b[i]| (NaN if any difference is
// NaN; an entry -inf in both counts 0). Non-negative floats order as their bit patterns,
// so the block maxima combine with an integer atomicMax on *out (zeroed by the caller).
__global__ void __launch_bounds__(256) k_residual(int64_t n, const float *__restrict__ a,
                                                  const float *__restrict__ b, unsigned *__restrict__ out) {
    float mx = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = __ldg(a + i), y = __ldg(b + i);
        const float dlt = (x == y) ? 0.f : fabsf(x - y);  // equal infinities: 0
        mx = (dlt != dlt || mx != mx) ? CUDART_NAN_F : fmaxf(mx, dlt);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const float o = __shfl_xor_sync(0xffffffffu, mx, d);
        mx = (o != o || mx != mx) ? CUDART_NAN_F : fmaxf(mx, o);
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(mx));  // NaN (0x7fc00000) ranks above +inf
}

// ---- per-member early exit of a batch ---------------------------------------------------

// Reset of a batched early-exit run: members with no edge-states are frozen from the
// start (0 iterations, residual 0), the others active; state[0] (iterations done) = 0.
__global__ void k_until_members_init(int32_t *__restrict__ frozen, unsigned *__restrict__ res,
                                     int32_t *__restrict__ iters, float *__restrict__ resid,
                                     const int32_t *__restrict__ off, int n_members, int *__restrict__ state) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n_members; m += gridDim.x * blockDim.x) {
        const bool empty = __ldg(off + m + 1) == __ldg(off + m);
        frozen[m] = empty ? 1 : 0;
        res[m] = 0u;
        iters[m] = 0;
        resid[m] = empty ? 0.f : CUDART_NAN_F;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) state[0] = 0;
}

// res[m] = max(res[m], max over member m's edge-states off[m]..off[m+1] of |a - b|), as
// k_residual, for members not frozen. A warp takes a contiguous run of edge-states
// (lanes interleaved, so loads coalesce); a lane adds its running maximum to the
// member's word when its member changes and at the end.
__global__ void __launch_bounds__(256) k_residual_members(int64_t n, const float *__restrict__ a,
                                                          const float *__restrict__ b,
                                                          const int32_t *__restrict__ off, int n_members,
                                                          const int32_t *__restrict__ frozen,
                                                          unsigned *__restrict__ res) {
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t chunk = (((n + n_warps - 1) / n_warps) + 31) & ~(int64_t)31;
    const int64_t i1 = min(n, (w + 1) * chunk);
    int64_t i = w * chunk + lane;
    if (i >= i1) return;
    int lo = 0, hi = n_members - 1;  // the member holding edge-state i: last m with off[m] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    int m = lo;
    int64_t end = __ldg(off + m + 1);
    float mx = 0.f;
    for (; i < i1; i += 32) {
        if (i >= end) {
            if (!__ldg(frozen + m)) atomicMax(res + m, __float_as_uint(mx));
            mx = 0.f;
            do {
                ++m;
                end = __ldg(off + m + 1);
            } while (i >= end);
        }
        const float x = __ldg(a + i), y = __ldg(b + i);
        const float dlt = (x == y) ? 0.f : fabsf(x - y);
        mx = (dlt != dlt || mx != mx) ? CUDART_NAN_F : fmaxf(mx, dlt);
    }
    if (!__ldg(frozen + m)) atomicMax(res + m, __float_as_uint(mx));
}

// Loop control of a batched early-exit run after a trip of n iterations (one block):
// state[0] += n; a member frozen last trip (2) becomes 1; an active member records its
// iterations and residual, and freezes (2: its messages are copied next) when the
// residual is <= tol; its residual word is reset for the next trip. state[1] = whether
// to go on: a member is active and fewer than limit iterations are done (also the
// condition of the while node when set_condition); state[2] = a member is active.
__global__ void __launch_bounds__(256) k_until_control_members(cudaGraphConditionalHandle h, bool set_condition,
                                                               unsigned *__restrict__ res, int32_t *__restrict__ frozen,
                                                               int32_t *__restrict__ iters, float *__restrict__ resid,
                                                               int n_members, int *__restrict__ state, int n,
                                                               int limit, float tol) {
    const int d = state[0] + n;
    int active = 0;
    for (int m = threadIdx.x; m < n_members; m += blockDim.x) {
        const int f = frozen[m];
        if (f == 2) frozen[m] = 1;
        if (f != 0) continue;
        const float r = __uint_as_float(res[m]);
        res[m] = 0u;
        iters[m] = d;
        resid[m] = r;
        if (r <= tol) frozen[m] = 2;  // (false for NaN)
        else active = 1;
    }
    active = __syncthreads_or(active);
    if (threadIdx.x == 0) {
        state[0] = d;
        const int go = active && d < limit;
        state[1] = go;
        state[2] = active;
        if (set_condition) cudaGraphSetConditional(h, go ? 1u : 0u);
    }
}

// Members frozen at the last control (2): their messages a copied to the other
// ping-pong buffer b, so that both hold the iteration the member stopped at.
__global__ void __launch_bounds__(256) k_freeze_copy(const int32_t *__restrict__ frozen, const int32_t *__restrict__ off,
                                                     int n_members, const float *__restrict__ a, float *__restrict__ b) {
    for (int m = 0; m < n_members; ++m) {
        if (__ldg(frozen + m) != 2) continue;
        const int64_t s0 = __ldg(off + m), s1 = __ldg(off + m + 1);
        for (int64_t i = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s1; i += (int64_t)gridDim.x * blockDim.x)
            b[i] = a[i];
    }
}

// The loop control of a device-side early-exit run (the body of a conditional while
// node): after a trip of n iterations, done += n; the loop goes on while the trip's
// residual (bits in *res) is above tol or NaN and fewer than limit iterations are done.
// Batch run with iteration counts per member: after `it` iterations, the members whose
// count is `it` stop (frozen; the factor pass skips them) and their messages are copied
// from the buffer that holds iteration `it` (a) to the other one (b), so that both hold
// their last iteration whichever buffer the run ends in.
__global__ void __launch_bounds__(256) k_batch_freeze(const int32_t *__restrict__ n_iters, int it, int n_members,
                                                      const int32_t *__restrict__ off, int32_t *__restrict__ frozen,
                                                      const float *__restrict__ a, float *__restrict__ b) {
    for (int m = 0; m < n_members; ++m) {
        if (__ldg(n_iters + m) != it) continue;
        if (blockIdx.x == 0 && threadIdx.x == 0) frozen[m] = 1;
        const int64_t s0 = __ldg(off + m), s1 = __ldg(off + m + 1);
        for (int64_t i = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s1; i += (int64_t)gridDim.x * blockDim.x)
            b[i] = a[i];
    }
}

__global__ void k_until_control(cudaGraphConditionalHandle h, const unsigned *__restrict__ res,
                                int *__restrict__ done, int n, int limit, float tol) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int d = *done + n;
    *done = d;
    const float r = __uint_as_float(*res);
    cudaGraphSetConditional(h, ((r > tol) || (r != r)) && d < limit ? 1u : 0u);
}

// =====================================================================================
// Small binary pairwise graphs: one block for the whole run (Plan::lr, 4-slot layout)
// =====================================================================================
//
// On a graph of up to a few thousand variables the log-ratio run is bound by its
// launches, not by memory: each pass is one short wave of blocks, two dependent launches
// per iteration plus the conversions around the run. Here one block (below) or a cluster
// of blocks (further below) does the whole run in one launch. The block: it converts the messages into log-ratios in shared memory (as
// k_lr_pack_slot4), forms its factors' table numbers in registers (as k_lr_params), runs
// every iteration with block barriers between the steps, and writes the messages back (as
// k_lr_unpack). Per iteration a variable pass (thread t owns variable t; the totals Dv in
// shared memory) and a factor pass (thread t owns factor t, or factors t and t + n_t when
// there are more factors than a block has threads, and keeps their slot pairs and table
// numbers in registers for the whole run), with a block barrier after each. A thread with
// two factors loads both factors' shared-memory inputs before it computes and stores
// either (a factor's slots belong to that factor alone), so their latencies overlap. The
// per-item arithmetic is that of k_var_slot4_lr and k_pair2_lr step for step, so the
// messages are bitwise those of the multi-launch run. A variable on the explicit-sum path
// (an infinite evidence entry or message) writes its four lam (lr_var_slow) to global
// memory, which the factor pass reads after the barrier. (A schedule with one barrier per
// iteration, each factor forming its variables' totals itself into a second copy of d,
// measured the same on a 10 x 10 grid and up to 1.9x slower on larger ones.)

// Prologue: the log-ratios of msgs into d, as k_lr_pack_slot4 (msgs through L2: the
// epilogue writes it).
__device__ __forceinline__ void lr_small_pack(const DevGraph &G, const float *m, float *d) {
    const int V = G.V;
    for (int v = threadIdx.x; v < V; v += blockDim.x) {
        const int4 t = __ldg(G.vin_tab4 + v);
        const int es[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            d[q * V + v] = es[q] >= 0 ? lr_encode(__ldcg(m + es[q]), __ldcg(m + es[q] + 1)) : 0.f;
        }
    }
}

// Epilogue: every edge's two entries from its slot of d, as k_lr_unpack.
__device__ __forceinline__ void lr_small_unpack(const DevGraph &G, const float *d, float *m) {
    for (int e = threadIdx.x; e < G.E; e += blockDim.x) {
        const float2 q = lr_decode(d[__ldg(G.lr_pos + e)]);
        m[2 * (size_t)e] = q.x;
        m[2 * (size_t)e + 1] = q.y;
    }
}

// Factor g's slot pair and table numbers, as k_lr_params.
struct LrSmallFactor {
    int2 p;
    float c, al, be;
};
__device__ __forceinline__ LrSmallFactor lr_small_factor(const DevGraph &G, const EnumSeg *segs, int n_seg,
                                                         const float *pot, int g, int F) {
    LrSmallFactor r{make_int2(0, 0), 0.f, 0.f, 0.f};
    if (g >= F) return r;
    r.p = __ldg(reinterpret_cast<const int2 *>(G.lr_pos) + g);
    const float4 t = lr_table(segs, n_seg, pot, g);
    const bool fin = isfinite(t.x) & isfinite(t.y) & isfinite(t.z) & isfinite(t.w);
    r.c = fin ? t.z - t.x : CUDART_NAN_F;
    r.al = t.w - t.z;
    r.be = t.y - t.x;
    return r;
}

// The factor update of k_pair2_lr from the variable-to-factor log-ratios l0, l1 and the
// stored messages mo0, mo1.
template <bool MAXP>
__device__ __forceinline__ float2 lr_small_update(const LrSmallFactor &f, const EnumSeg *segs, int n_seg,
                                                  const float *pot, int g, float l0, float l1, float mo0,
                                                  float mo1, float k, float Tln2, float damping, float w,
                                                  uint32_t *flags) {
    const float dt0 = f.c + softplus_t<MAXP>(f.al + l1, k, Tln2) - softplus_t<MAXP>(f.be + l1, k, Tln2);
    const float dt1 = f.be + softplus_t<MAXP>(f.al + f.c - f.be + l0, k, Tln2) - softplus_t<MAXP>(f.c + l0, k, Tln2);
    float2 dn = make_float2(fmaf(damping, mo0, w * dt0), fmaf(damping, mo1, w * dt1));
    if (!(isfinite(dn.x) && isfinite(dn.y) && l0 == l0 && l1 == l1)) {
        const float4 t = lr_table(segs, n_seg, pot, g);
        const float t4[4] = {t.x, t.y, t.z, t.w};
        dn = pair2_lr_exact<MAXP>(t4, l0, l1, mo0, mo1, k, Tln2, damping, flags);
    }
    return dn;
}

// The variable pass of k_var_slot4_lr for one variable: its total into *Dv, or kDvSlow
// and its four lam (lr_var_slow) into global lam.
__device__ __forceinline__ void lr_small_var(float2 e, const float (&dk)[4], int v, int V, float2 *Dv,
                                             float *lam) {
    bool fin = isfinite(e.x) & isfinite(e.y);
#pragma unroll
    for (int q = 0; q < 4; ++q) fin &= isfinite(dk[q]);
    if (fin) {
        FF D = ff_add_nc(ff_make(e.y), -e.x);
#pragma unroll
        for (int q = 0; q < 4; ++q) D = ff_add_nc(D, dk[q]);
        const float2 Df = make_float2(D.hi, D.lo);
        bool ok = true;
#pragma unroll
        for (int q = 0; q < 4; ++q) ok &= isfinite(lr_lam_from_D(Df, dk[q]));
        if (ok) {
            *Dv = Df;
            return;
        }
    }
    const int pos[4] = {v, V + v, 2 * V + v, 3 * V + v};
    lr_var_slow(e, dk, pos, 4, lam);
    *Dv = make_float2(__uint_as_float(kDvSlow), 0.f);
}

template <bool MAXP, int NF>
__global__ void __launch_bounds__(kLrSmallThreads)
k_lr_small(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
            const float *__restrict__ ev, float *__restrict__ msgs, float *__restrict__ lam, float k, float Tln2,
            float damping, int n_iters) {
    extern __shared__ __align__(16) float lr_sm[];
    const int V = G.V, F = G.E / 2, tid = threadIdx.x, nt = blockDim.x;
    float2 *Dv = reinterpret_cast<float2 *>(lr_sm);  // V float2 (8-byte aligned at the base)
    float *d = lr_sm + 2 * (size_t)V;                // 4 V floats
    lr_small_pack(G, msgs, d);
    const float2 e = tid < V ? __ldg(reinterpret_cast<const float2 *>(ev) + tid) : make_float2(0.f, 0.f);
    LrSmallFactor f[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) f[j] = lr_small_factor(G, segs, n_seg, pot, tid + j * nt, F);
    const float w = 1.f - damping;
    __syncthreads();
    for (int it = 0; it < n_iters; ++it) {
        if (tid < V) {  // variable pass (k_var_slot4_lr)
            float dk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) dk[q] = d[q * V + tid];
            lr_small_var(e, dk, tid, V, Dv + tid, lam);
        }
        __syncthreads();
        float mo0[NF], mo1[NF];  // factor pass (k_pair2_lr<MAXP, true>)
        float2 D0[NF], D1[NF];
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const int2 p = f[j].p;
            mo0[j] = d[p.x];
            mo1[j] = d[p.y];
            D0[j] = Dv[p.x - V * ((p.x >= V) + (p.x >= 2 * V) + (p.x >= 3 * V))];
            D1[j] = Dv[p.y - V * ((p.y >= V) + (p.y >= 2 * V) + (p.y >= 3 * V))];
        }
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const int g = tid + j * nt;
            if (g >= F) continue;
            const int2 p = f[j].p;
            const float l0 = __float_as_uint(D0[j].x) == kDvSlow ? __ldcg(lam + p.x) : lr_lam_from_D(D0[j], mo0[j]);
            const float l1 = __float_as_uint(D1[j].x) == kDvSlow ? __ldcg(lam + p.y) : lr_lam_from_D(D1[j], mo1[j]);
            const float2 dn = lr_small_update<MAXP>(f[j], segs, n_seg, pot, g, l0, l1, mo0[j], mo1[j], k, Tln2,
                                                    damping, w, G.flags);
            d[p.x] = dn.x;
            d[p.y] = dn.y;
        }
        __syncthreads();
    }
    lr_small_unpack(G, d, msgs);
}

// ---- a cluster of blocks: graphs of up to 16,384 variables -----------------------------
//
// Above one block's share the same run goes to a thread-block cluster of C blocks
// (lr_cluster_size: 16 or 8; co-scheduled, one per SM) whose shared memories together hold d and the totals D,
// distributed by variable: block r owns variables r Vc .. (r + 1) Vc - 1 (their four slots,
// plane q at q Vc, and their totals) and factors r Fc .. (r + 1) Fc - 1. A factor reads and
// writes its two slots, and reads its variables' totals, in whichever block holds them,
// through the cluster's distributed shared memory (mapa: the generic address of the same
// offset in another block). The passes are separated by cluster barriers (arrive with
// release, wait with acquire, at cluster scope: they also order the explicit-sum path's
// global lam), and a block leaves only after a last barrier, once no block reads another's
// memory. Every thread of every block runs every barrier. The per-item arithmetic is that
// of the multi-launch kernels, so the messages are bitwise theirs.

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// The generic address of the same shared-memory location in block `rank` of the cluster.
template <class Tp>
__device__ __forceinline__ Tp *rank_ptr(Tp *p, uint32_t rank) {
    uint64_t out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<Tp *>(out);
}

// Slot p = k V + v of the 4-slot layout: the block that owns v and the slot's offset in its
// d (k Vc + the variable's local index); also the local index of the variable.
__device__ __forceinline__ void lr_slot_home(int p, int V, int Vc, uint32_t &rank, int &off, int &lv) {
    const int k = (p >= V) + (p >= 2 * V) + (p >= 3 * V);
    const int v = p - k * V;
    rank = (uint32_t)(v / Vc);
    lv = v - (int)rank * Vc;
    off = k * Vc + lv;
}

template <bool MAXP, int NF>
__global__ void __launch_bounds__(kLrSmallThreads)
k_lr_cluster(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
             const float *__restrict__ ev, float *__restrict__ msgs, float *__restrict__ lam, float k, float Tln2,
             float damping, int n_iters, int Vc, int Fc) {
    extern __shared__ __align__(16) float lr_sm[];
    const int V = G.V, F = G.E / 2, tid = threadIdx.x, nt = blockDim.x;
    const uint32_t r = cluster_rank();
    float2 *Dv = reinterpret_cast<float2 *>(lr_sm);  // Vc float2: this block's variables' totals
    float *d = lr_sm + 2 * (size_t)Vc;               // 4 Vc floats: their slots
    const int v0 = (int)r * Vc, nv = max(0, min(Vc, V - v0));
    // this block's variables' slots from msgs (as k_lr_pack_slot4)
    for (int lv = tid; lv < nv; lv += nt) {
        const int4 t = __ldg(G.vin_tab4 + v0 + lv);
        const int es[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            d[q * Vc + lv] = es[q] >= 0 ? lr_encode(__ldcg(msgs + es[q]), __ldcg(msgs + es[q] + 1)) : 0.f;
    }
    const bool hv = tid < nv;
    const float2 e = hv ? __ldg(reinterpret_cast<const float2 *>(ev) + v0 + tid) : make_float2(0.f, 0.f);
    // this thread's factors: table numbers and where their slots and totals live
    LrSmallFactor f[NF];
    float *s0[NF], *s1[NF];
    const float2 *t0[NF], *t1[NF];
    bool hf[NF];
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const int i = tid + j * nt, g = (int)r * Fc + i;
        hf[j] = i < Fc && g < F;
        f[j] = lr_small_factor(G, segs, n_seg, pot, hf[j] ? g : F, F);  // (0, 0) for no factor
        uint32_t ra, rb;
        int oa, ob, la, lb;
        lr_slot_home(f[j].p.x, V, Vc, ra, oa, la);
        lr_slot_home(f[j].p.y, V, Vc, rb, ob, lb);
        s0[j] = rank_ptr(d + oa, ra);
        s1[j] = rank_ptr(d + ob, rb);
        t0[j] = rank_ptr(Dv + la, ra);
        t1[j] = rank_ptr(Dv + lb, rb);
    }
    const float w = 1.f - damping;
    cluster_barrier();  // every block's slots are packed
    for (int it = 0; it < n_iters; ++it) {
        if (hv) {  // variable pass (k_var_slot4_lr), this block's variables
            float dk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) dk[q] = d[q * Vc + tid];
            lr_small_var(e, dk, v0 + tid, V, Dv + tid, lam);
        }
        cluster_barrier();
        float mo0[NF], mo1[NF];  // factor pass (k_pair2_lr<MAXP, true>), this block's factors
        float2 D0[NF], D1[NF];
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            mo0[j] = *s0[j];
            mo1[j] = *s1[j];
            D0[j] = *t0[j];
            D1[j] = *t1[j];
        }
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            if (!hf[j]) continue;
            const int2 p = f[j].p;
            const float l0 = __float_as_uint(D0[j].x) == kDvSlow ? __ldcg(lam + p.x) : lr_lam_from_D(D0[j], mo0[j]);
            const float l1 = __float_as_uint(D1[j].x) == kDvSlow ? __ldcg(lam + p.y) : lr_lam_from_D(D1[j], mo1[j]);
            const float2 dn = lr_small_update<MAXP>(f[j], segs, n_seg, pot, (int)r * Fc + tid + j * nt, l0, l1,
                                                    mo0[j], mo1[j], k, Tln2, damping, w, G.flags);
            *s0[j] = dn.x;
            *s1[j] = dn.y;
        }
        cluster_barrier();
    }
    // the edges of this block's factors back into msgs (as k_lr_unpack)
    const int e_end = 2 * min(F, ((int)r + 1) * Fc);
    for (int ei = 2 * (int)r * Fc + tid; ei < e_end; ei += nt) {
        uint32_t ra;
        int oa, la;
        lr_slot_home(__ldg(G.lr_pos + ei), V, Vc, ra, oa, la);
        const float2 q = lr_decode(*rank_ptr(d + oa, ra));
        msgs[2 * (size_t)ei] = q.x;
        msgs[2 * (size_t)ei + 1] = q.y;
    }
    cluster_barrier();  // no block leaves while another may still read its shared memory
}

}  // namespace

// =====================================================================================
// Launchers
// =====================================================================================

cudaError_t prepare_kernels(int max_smem_bytes);

// Blocks of k_enum_block resident on one SM at `threads` threads and `smem` bytes of
// dynamic shared memory: the smaller count of its max-product and sum-product forms
// (at least 1).
int enum_block_resident(int threads, int smem) {
    if (smem > 48 * 1024 && prepare_kernels(smem) != cudaSuccess) return 1;
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_enum_block<true, false>, threads, (size_t)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_enum_block<false, false>, threads, (size_t)smem) !=
            cudaSuccess)
        return 1;
    return std::max(1, std::min(a, b));
}

// The kernels with dynamic shared memory may take up to the device's opt-in maximum
// (set once per device; a smaller limit set later would break other graphs' launches;
// two threads that race here both set the same values).
cudaError_t prepare_kernels(int max_smem_bytes) {
    static volatile int done[64];
    if (max_smem_bytes <= 48 * 1024) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    // each kernel: the opt-in maximum less its static shared memory
    auto allow = [&](const void *fn) -> cudaError_t {
        cudaFuncAttributes fa{};
        cudaError_t r = cudaFuncGetAttributes(&fa, fn);
        if (r != cudaSuccess) return r;
        const int dyn = optin - (int)fa.sharedSizeBytes;
        if (max_smem_bytes > dyn) return cudaErrorInvalidValue;
        return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    };
    if ((e = allow((const void *)k_logic_warp<true>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_logic_warp<false>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_enum_block<true>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_enum_block<false>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_logic_warp<true, true>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_logic_warp<false, true>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_enum_block<true, true>)) != cudaSuccess) return e;
    if ((e = allow((const void *)k_enum_block<false, true>)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = 1;
    return cudaSuccess;
}

// Launches a kernel of the iteration or the adjoint chain with the programmatic
// attribute: its launch and block dispatch overlap the previous kernel's last blocks, and
// the kernel itself waits (pdl_wait) before it touches global memory.
template <typename... KArgs, typename... Args>
static void launch_dep(void (*kernel)(KArgs...), dim3 grid, int threads, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);  // errors surface through cudaGetLastError
}

template <int MODE, bool MS>
static void var_pass_mode(const DevGraph &G, const Plan &P, const float *ev, const float *m,
                          float *out, int32_t *dec, cudaStream_t s, int S, const LaunchHook *hook) {
    if (G.vin_tab4 != nullptr) {
        const int n = G.V;
        k_var_tab4<MODE, MS><<<dim3((n + 255) / 256, S), 256, 0, s>>>(G, n, ev, m, out, dec);
        if (hook) hook->after(hook->ctx);
        return;
    }
    for (const VarLaunch &L : P.var) {
        if (L.n == 0) continue;
        switch (L.kind) {
            case kVarBlock:  // single-sample launches: a block per tile; else a block per variable
                if (!MS && S == 1 && L.tiles != nullptr && G.hd_tot != nullptr && G.hd_cnt != nullptr)
                    launch_dep(k_var_hd<MODE>, dim3(L.n_tiles), kVarBlockThreads, 0, s, G, L.list, L.tiles, ev, m, out, dec);
                else
                    launch_dep(k_var_block<MODE, MS>, dim3(dim3(L.n, S)), kVarBlockThreads, 0, s, G, L.list, ev, m, out, dec);
                break;
            case kVarBinary:
                launch_dep(k_var_thread<2, MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, L.dense_binary, ev, m, out, dec);
                break;
            case kVarGroup4:
                launch_dep(k_var_group<4, MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, ev, m, out, dec);
                break;
            case kVarGroup8:
                launch_dep(k_var_group<8, MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, ev, m, out, dec);
                break;
            case kVarGroup16:
                launch_dep(k_var_group<16, MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, ev, m, out, dec);
                break;
            case kVarWarp:
                launch_dep(k_var_warp<MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, ev, m, out, dec);
                break;
            default:
                launch_dep(k_var_thread<0, MODE, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, L.list, L.n, 0, ev, m, out, dec);
                break;
        }
        if (hook) hook->after(hook->ctx);
    }
}

cudaError_t launch_var_pass(const DevGraph &G, const Plan &P, const float *ev, const float *m,
                            float *b, int mode, int32_t *decode, cudaStream_t s, int S, const LaunchHook *hook) {
    if (mode == kVarIter && S > 1) var_pass_mode<kVarIter, true>(G, P, ev, m, b, decode, s, S, hook);
    else if (mode == kVarIter) var_pass_mode<kVarIter, false>(G, P, ev, m, b, decode, s, 1, hook);
    else if (mode == kVarBeliefs) var_pass_mode<kVarBeliefs, false>(G, P, ev, m, b, decode, s, 1, hook);
    else if (mode == kVarNormalised) var_pass_mode<kVarNormalised, false>(G, P, ev, m, b, decode, s, 1, hook);
    else var_pass_mode<kVarDecode, false>(G, P, ev, m, b, decode, s, 1, hook);
    return cudaGetLastError();
}

template <bool MAXP, bool MS>
static void factor_pass_t(const DevGraph &G, const Plan &P, const float *pot, const float *b,
                          const float *ev, const float *m_old, float *m_new, float T, float damping,
                          cudaStream_t s, int S, const LaunchHook *hook) {
    const float invT = MAXP ? 0.f : 1.f / T;
    for (const FactorLaunch &L : P.factor) {
        if (L.n_blocks == 0) continue;
        const EnumSeg *es = static_cast<const EnumSeg *>(L.segs);
        const LogicSeg *ls = static_cast<const LogicSeg *>(L.segs);
        switch (L.variant) {
            case kPair2:
                launch_dep(k_pair<2, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair4:
                k_pair_group<4, MAXP, MS><<<dim3(min(L.n_blocks, L.max_blocks), S), L.threads, 0, s>>>(G, es, L.n_seg, L.n_blocks, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair8:
                k_pair_group<8, MAXP, MS><<<dim3(min(L.n_blocks, L.max_blocks), S), L.threads, 0, s>>>(G, es, L.n_seg, L.n_blocks, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair16:
                k_pair_group<16, MAXP, MS><<<dim3(min(L.n_blocks, L.max_blocks), S), L.threads, 0, s>>>(G, es, L.n_seg, L.n_blocks, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairT4:
                launch_dep(k_pair_thr<4, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairT8:
                launch_dep(k_pair_thr<8, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairT16:
                launch_dep(k_pair_thr<16, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairD4:
                launch_dep(k_pair_dir<4, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairD8:
                launch_dep(k_pair_dir<8, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairD16:
                launch_dep(k_pair_dir<16, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairQ8:
                launch_dep(k_pair_quad<8, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPairQ16:
                launch_dep(k_pair_quad<16, MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kEnumGeneric:
                launch_dep(k_enum_generic<MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kEnumBlock:
                launch_dep(k_enum_block<MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, L.smem, s, G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kLogicSmall:
                if (L.max_fan <= 2)
                    launch_dep(k_logic_small<MAXP, MS, 2>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, ls, L.n_seg, b, ev, m_old, m_new, T, invT, damping);
                else
                    launch_dep(k_logic_small<MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, 0, s, G, ls, L.n_seg, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kLogicWarp:
                launch_dep(k_logic_warp<MAXP, MS>, dim3(dim3(L.n_blocks, S)), L.threads, L.smem, s, G, ls, L.n_seg, b, ev, m_old, m_new, T, invT, damping, L.max_fan);
                break;
            default:
                break;
        }
        if (hook) hook->after(hook->ctx);
    }
}

// A launch that may begin while the previous kernel of the stream finishes (the kernel
// waits for it with pdl_wait before touching its output).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int blocks, int threads, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

cudaError_t launch_lr_var_pass(const DevGraph &G, const Plan &P, const float *ev, const float *d, float2 *Dv,
                               float *lam, cudaStream_t s, const LaunchHook *hook) {
    cudaError_t e = cudaSuccess;
    if (G.vin_tab4 != nullptr) {
        e = launch_pdl(k_var_slot4_lr, (G.V + 255) / 256, 256, s, G.V, ev, d, Dv, lam);
        if (hook && e == cudaSuccess) hook->after(hook->ctx);
    } else {
        for (const VarLaunch &L : P.var)
            if (L.n > 0 && e == cudaSuccess) {
                e = launch_pdl(k_var_csr_lr, L.n_blocks, L.threads, s, G, L.list, L.n, ev, d, lam);
                if (hook && e == cudaSuccess) hook->after(hook->ctx);
            }
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lr_params(const DevGraph &G, const Plan &P, const float *log_pot, float *prm, cudaStream_t s) {
    const int F = G.E / 2;
    for (const FactorLaunch &L : P.factor) {  // the one kPair2 launch: every factor
        if (L.n_blocks == 0 || F == 0) continue;
        k_lr_params<<<(F + 255) / 256, 256, 0, s>>>(static_cast<const EnumSeg *>(L.segs), L.n_seg, F, log_pot, prm);
    }
    return cudaGetLastError();
}

cudaError_t launch_lr_factor_pass(const DevGraph &G, const Plan &P, const float *log_pot, const float *prm,
                                  const float2 *Dv, const float *lam, float *d, float T, float damping,
                                  cudaStream_t s, const LaunchHook *hook) {
    // lse2_fast constants: k = log2(e) / T, T ln 2
    const float k = T > 0.f ? (float)(1.4426950408889634 / (double)T) : 0.f;
    const float Tln2 = (float)((double)T * 0.6931471805599453);
    const int2 *pos2 = reinterpret_cast<const int2 *>(G.lr_pos);
    const int F = G.E / 2;
    for (const FactorLaunch &L : P.factor) {  // the one kPair2 launch: every factor
        if (L.n_blocks == 0) continue;
        const EnumSeg *es = static_cast<const EnumSeg *>(L.segs);
        // persistent: as many blocks of 256 as are resident at once (8 per SM), or fewer
        const int blocks = std::min<int>(P.lr_blocks, (F + 255) / 256);
        const bool from_d = G.vin_tab4 != nullptr;
        auto kern = T == 0.f ? (from_d ? k_pair2_lr<true, true> : k_pair2_lr<true, false>)
                             : (from_d ? k_pair2_lr<false, true> : k_pair2_lr<false, false>);
        cudaError_t e = launch_pdl(kern, blocks, 256, s, es, L.n_seg, F, G.V, pos2, (const float *)prm, log_pot,
                                   Dv, lam, d, G.flags, k, Tln2, damping);
        if (e != cudaSuccess) return e;
        if (hook) hook->after(hook->ctx);
    }
    return cudaGetLastError();
}

cudaError_t launch_ms_prepare(const DevGraph &G, const Plan &P, int S, int Sp, int64_t n_pot,
                              const float *log_pot, const float *ev, const float *msgs, float2 *ev_s, float *d,
                              float *prm, cudaStream_t s) {
    const int64_t nv = (int64_t)G.V * S, F = G.E / 2;
    k_ms_evidence<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(G.V, S, G.VS, ev, ev_s);
    k_ms_pack<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(G, S, msgs, d);
    for (const FactorLaunch &L : P.factor)  // the one kPair2 launch: every factor
        if (L.n_blocks > 0 && F > 0)
            k_ms_params<<<(unsigned)((F * Sp + 255) / 256), 256, 0, s>>>(static_cast<const EnumSeg *>(L.segs),
                                                                        L.n_seg, (int)F, Sp, n_pot, log_pot, prm);
    return cudaGetLastError();
}

cudaError_t launch_ms_iteration(const DevGraph &G, const Plan &P, int S, int Sp, int64_t n_pot,
                                const float *log_pot, const float *prm, const float2 *ev_s, float *d, float2 *Dv,
                                float *lam, float T, float damping, cudaStream_t s) {
    const int64_t nv = (int64_t)G.V * S, F = G.E / 2;
    cudaError_t e = launch_pdl(k_ms_var, (int)((nv + 255) / 256), 256, s, G.V, S, ev_s, (const float *)d, Dv, lam);
    if (e != cudaSuccess) return e;
    const float k = T > 0.f ? (float)(1.4426950408889634 / (double)T) : 0.f;
    const float Tln2 = (float)((double)T * 0.6931471805599453);
    const int2 *pos2 = reinterpret_cast<const int2 *>(G.lr_pos);
    for (const FactorLaunch &L : P.factor) {
        if (L.n_blocks == 0) continue;
        const EnumSeg *es = static_cast<const EnumSeg *>(L.segs);
        const int blocks = (int)std::min<int64_t>(P.lr_blocks, (F * S + 255) / 256);
        auto kern = T == 0.f ? k_ms_pair<true> : k_ms_pair<false>;
        e = launch_pdl(kern, blocks, 256, s, es, L.n_seg, (int)F, G.V, S, Sp, n_pot, pos2, prm, log_pot,
                       (const float2 *)Dv, (const float *)lam, d, G.flags, k, Tln2, damping);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_until_members_init(int32_t *frozen, unsigned *res, int32_t *iters, float *resid,
                                      const int32_t *off, int n_members, int *state, cudaStream_t s) {
    k_until_members_init<<<std::max(1, std::min((n_members + 255) / 256, 1024)), 256, 0, s>>>(frozen, res, iters, resid,
                                                                                              off, n_members, state);
    return cudaGetLastError();
}

cudaError_t launch_residual_members(int64_t n, const float *a, const float *b, const int32_t *off, int n_members,
                                    const int32_t *frozen, unsigned *res, int n_sm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 8);
    k_residual_members<<<blocks, 256, 0, s>>>(n, a, b, off, n_members, frozen, res);
    return cudaGetLastError();
}

cudaError_t launch_until_control_members(cudaGraphConditionalHandle h, bool set_condition, unsigned *res,
                                         int32_t *frozen, int32_t *iters, float *resid, int n_members, int *state,
                                         int n, int limit, float tol, cudaStream_t s) {
    k_until_control_members<<<1, 256, 0, s>>>(h, set_condition, res, frozen, iters, resid, n_members, state, n, limit,
                                              tol);
    return cudaGetLastError();
}

cudaError_t launch_freeze_copy(const int32_t *frozen, const int32_t *off, int n_members, const float *a, float *b,
                               int n_sm, cudaStream_t s) {
    k_freeze_copy<<<n_sm * 4, 256, 0, s>>>(frozen, off, n_members, a, b);
    return cudaGetLastError();
}

cudaError_t launch_batch_freeze(const int32_t *n_iters, int it, int n_members, const int32_t *off, int32_t *frozen,
                                const float *a, float *b, int n_sm, cudaStream_t s) {
    k_batch_freeze<<<n_sm * 4, 256, 0, s>>>(n_iters, it, n_members, off, frozen, a, b);
    return cudaGetLastError();
}

cudaError_t launch_residual(int64_t n, const float *a, const float *b, unsigned *out, int n_sm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)std::min<int64_t>(want, (int64_t)n_sm * 8);
    k_residual<<<blocks, 256, 0, s>>>(n, a, b, out);
    return cudaGetLastError();
}

cudaError_t launch_until_control(cudaGraphConditionalHandle h, const unsigned *res, int *done, int n, int limit,
                                 float tol, cudaStream_t s) {
    k_until_control<<<1, 32, 0, s>>>(h, res, done, n, limit, tol);
    return cudaGetLastError();
}

cudaError_t launch_pmp_perturb(int64_t VS, int S, const float *ev, const float *noise, float *out, cudaStream_t s) {
    const int64_t n = VS * S;
    if (n > 0) k_pmp_perturb<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(VS, S, ev, noise, out);
    return cudaGetLastError();
}

cudaError_t launch_ms_unpack(const DevGraph &G, int S, const float *d, float *msgs, cudaStream_t s) {
    const int64_t n = (int64_t)G.E * S;
    if (n > 0) k_ms_unpack<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G, S, d, msgs);
    return cudaGetLastError();
}

cudaError_t launch_lr_pack(const DevGraph &G, const float *m, float *d, cudaStream_t s) {
    if (G.E <= 0) return cudaSuccess;
    if (G.vin_tab4 != nullptr) k_lr_pack_slot4<<<(G.V + 255) / 256, 256, 0, s>>>(G, m, d);
    else k_lr_pack_csr<<<(G.E + 255) / 256, 256, 0, s>>>(G, m, d);
    return cudaGetLastError();
}

cudaError_t launch_lr_unpack(const DevGraph &G, const float *d, float *m, cudaStream_t s) {
    if (G.E <= 0) return cudaSuccess;
    const int blocks = (G.E + 255) / 256;
    if ((reinterpret_cast<uintptr_t>(m) & 7u) == 0) k_lr_unpack<true><<<blocks, 256, 0, s>>>(G, d, m);
    else k_lr_unpack<false><<<blocks, 256, 0, s>>>(G, d, m);
    return cudaGetLastError();
}

// The cluster size of the cluster form on this device: 16 blocks of kLrSmallThreads threads
// where the device places such a cluster (above the portable size of 8), else 8, else 0
// (asked once per device).
int lr_cluster_size() {
    static int size[64];  // 0 unknown, else the size + 1
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (size[dev] == 0) {
        void (*kerns[4])(DevGraph, const EnumSeg *, int, const float *, const float *, float *, float *, float,
                         float, float, int, int, int) = {k_lr_cluster<false, 1>, k_lr_cluster<false, 2>,
                                                         k_lr_cluster<true, 1>, k_lr_cluster<true, 2>};
        for (auto kern : kerns) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        int found = 0;
        for (int C : {kLrClusterMax, 8}) {
            cudaLaunchConfig_t cfg{};
            cfg.gridDim = dim3(C);
            cfg.blockDim = dim3(kLrSmallThreads);
            cfg.dynamicSmemBytes = (size_t)24 * kLrSmallMaxV;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            bool yes = true;
            for (auto kern : kerns) {
                int n = 0;
                yes = yes && cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
            }
            cudaGetLastError();  // a refused query leaves no error behind
            if (yes) {
                found = C;
                break;
            }
        }
        size[dev] = found + 1;
    }
    return size[dev] - 1;
}

cudaError_t launch_lr_small_run(const DevGraph &G, const Plan &P, const float *log_pot, const float *ev,
                                float *msgs, float *lam, float T, float damping, int n_iters, bool cluster,
                                cudaStream_t s) {
    const float k = T > 0.f ? (float)(1.4426950408889634 / (double)T) : 0.f;
    const float Tln2 = (float)((double)T * 0.6931471805599453);
    const int F = G.E / 2, V = G.V;
    const bool block = !cluster;
    if (!(block ? lr_block_fits(V, F) : lr_cluster_fits(V, F)) || G.vin_tab4 == nullptr || G.lr_pos == nullptr)
        return cudaErrorInvalidValue;
    for (const FactorLaunch &L : P.factor) {  // the one kPair2 launch: every factor
        if (L.n_blocks == 0 || n_iters <= 0) continue;
        const EnumSeg *segs = static_cast<const EnumSeg *>(L.segs);
        if (block) {  // one block: one variable and one factor per thread, or two factors
            const bool one = F <= kLrSmallThreads;
            const int per = one ? std::max(V, F) : std::max(V, (F + 1) / 2);
            const int threads = std::max(32, ((per + 31) / 32) * 32);
            const size_t smem = (size_t)V * 6 * sizeof(float);
            auto kern = T == 0.f ? (one ? k_lr_small<true, 1> : k_lr_small<true, 2>)
                                 : (one ? k_lr_small<false, 1> : k_lr_small<false, 2>);
            kern<<<1, threads, smem, s>>>(G, segs, L.n_seg, log_pot, ev, msgs, lam, k, Tln2, damping, n_iters);
            continue;
        }
        // a cluster of C blocks: block r owns Vc variables and Fc factors
        const int C = lr_cluster_size();
        const int Vc = (V + C - 1) / C, Fc = (F + C - 1) / C;
        const bool one = Fc <= kLrSmallThreads;
        const int per = one ? std::max(Vc, Fc) : std::max(Vc, (Fc + 1) / 2);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(std::max(32, ((per + 31) / 32) * 32));
        cfg.dynamicSmemBytes = (size_t)Vc * 6 * sizeof(float);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        auto kern = T == 0.f ? (one ? k_lr_cluster<true, 1> : k_lr_cluster<true, 2>)
                             : (one ? k_lr_cluster<false, 1> : k_lr_cluster<false, 2>);
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, G, segs, L.n_seg, log_pot, ev, msgs, lam, k, Tln2, damping,
                                           n_iters, Vc, Fc);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_factor_pass(const DevGraph &G, const Plan &P, const float *log_pot,
                               const float *b, const float *ev, const float *m_old,
                               float *m_new, float T, float damping, cudaStream_t s, int S,
                               const LaunchHook *hook) {
    if (S > 1) {  // the multi-sample instantiations
        if (T == 0.f) factor_pass_t<true, true>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s, S, hook);
        else factor_pass_t<false, true>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s, S, hook);
    } else {
        if (T == 0.f) factor_pass_t<true, false>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s, 1, hook);
        else factor_pass_t<false, false>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s, 1, hook);
    }
    return cudaGetLastError();
}

}  // namespace pgm

namespace pgm {

cudaError_t launch_adj_beliefs(const DevGraph &G, const float *ev, const float *m, const float *gnb, float *d_ev,
                               float *adj, cudaStream_t s) {
    launch_dep(k_adj_beliefs, dim3((G.V + 127) / 128), 128, 0, s, G, ev, m, gnb, d_ev, adj);
    return cudaGetLastError();
}

cudaError_t launch_adj_factor(const DevGraph &G, const FactorLaunch &L, const float *pot, const float *b,
                              const float *ev, const float *m_old, const float *adj, float *dv2f, float *ddamp,
                              float *d_pot, float *partials, int nc_max, float T, float damping, cudaStream_t s) {
    if (L.n_blocks == 0) return cudaSuccess;
    if (L.variant == kEnumBlock) {
        launch_dep(k_adj_block, dim3(L.n_blocks), L.threads, L.smem, s, G, static_cast<const EnumSeg *>(L.segs), L.n_seg, pot, b, ev,
                   m_old, adj, dv2f, ddamp, d_pot, partials, nc_max, T, 1.f / T, damping);
        if (partials != nullptr)
            launch_dep(k_adj_block_reduce, dim3(L.n_seg), 256, 0, s, static_cast<const EnumSeg *>(L.segs), L.n_seg,
                       partials, nc_max, d_pot);
    } else {
        launch_dep(k_adj_factor, dim3(L.n_blocks), L.threads, 0, s, G, static_cast<const EnumSeg *>(L.segs), L.n_seg, pot, b, ev,
                                                      m_old, adj, dv2f, ddamp, d_pot, partials, nc_max, T, 1.f / T,
                                                      damping);
        if (partials != nullptr)
            launch_dep(k_adj_pot_reduce, dim3(L.n_seg), 256, 0, s, static_cast<const EnumSeg *>(L.segs), L.n_seg, partials, nc_max,
                                                     L.threads, d_pot);
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_logic(const DevGraph &G, const FactorLaunch &L, const float *b, const float *ev,
                             const float *m_old, const float *adj, float *dv2f, float *ddamp, float T, float damping,
                             cudaStream_t s) {
    if (L.n_blocks == 0) return cudaSuccess;
    launch_dep(k_adj_logic, dim3(L.n_blocks), L.threads, 0, s, G, static_cast<const LogicSeg *>(L.segs), L.n_seg, b, ev, m_old, adj,
                                                 dv2f, ddamp, T, damping);
    return cudaGetLastError();
}

cudaError_t launch_adj_var(const DevGraph &G, const float *ddamp, const float *dv2f, float *adj_prev, float *d_ev,
                           cudaStream_t s) {
    if (G.vin_tab4 != nullptr) launch_dep(k_adj_var_tab4, dim3((G.V + 63) / 64), 64, 0, s, G, ddamp, dv2f, adj_prev, d_ev);
    else launch_dep(k_adj_var, dim3((G.V + 127) / 128), 128, 0, s, G, ddamp, dv2f, adj_prev, d_ev);
    return cudaGetLastError();
}

}  // namespace pgm
