// CUDA kernels (sm_103a) of one flooding LBP iteration and of the belief read-out.
//
// Method (PGMax, arXiv 2202.04110): log-space loopy belief propagation with parallel
// updates and damping (Sec. 3), enumeration factors over listed configurations
// (Sec. 4.2), OR / AND factors with updates linear in the fan-in (Sec. 3), flat
// message arrays updated by gather / scatter (Sec. 4), MAP decode (Sec. 4.1).
//
// One iteration is two passes over HBM-resident flat arrays:
//   variable pass  b_v = e_v + sum_{f in N(v)} m_{f->v}            (k_var_*)
//   factor pass    m_{v->f} = b_v - m_{f->v}   (gathered per edge)
//                  mt_{f->i} = factor update (LSE_T over configurations, or the
//                              closed-form OR / AND update)
//                  m_{f->i} <- norm(delta * m_{f->i} + (1 - delta) * norm(mt_{f->i}))
//                  written to the other buffer of a ping-pong pair   (k_pair, k_enum_generic,
//                                                                     k_logic_small, k_logic_warp)
// The path is gather / scatter plus log-sum-exp, bound by HBM bandwidth (or by the SFU
// for large state counts), not a dense contraction: no tensor cores.
//
// Numerics: messages, beliefs and all arithmetic in FP32. When a stored message entry
// is -inf the subtraction b - m would be -inf - (-inf); that entry's leave-one-out sum
// is then recomputed explicitly from the variable's incoming messages (v2f_slow).
#include <cstdint>

#include <cuda_runtime.h>
#include <math_constants.h>

#include "pgm_internal.h"

namespace pgm {
namespace {

constexpr uint32_t kFlagContradiction = 1u;
constexpr uint32_t kFlagNaN = 2u;

#define kNegInf (-CUDART_INF_F)
__device__ __forceinline__ float pos_inf() { return CUDART_INF_F; }

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

// ---- variable-to-factor value -------------------------------------------------------

// Explicit leave-one-out sum e_v(x) + sum over incoming edges other than `es`; used only
// when the edge's own message entry is -inf (rare: hard constraints).
__device__ __noinline__ float v2f_slow(const DevGraph G, const float *__restrict__ ev,
                                       const float *__restrict__ m, int vs, int es, int x) {
    int lo = 0, hi = G.V - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (G.vs_off[mid] <= vs) lo = mid;
        else hi = mid - 1;
    }
    float s = ev[vs + x];
    for (int k = G.vin_off[lo]; k < G.vin_off[lo + 1]; ++k) {
        int e2 = G.vin_es[k];
        if (e2 != es) s += m[e2 + x];
    }
    return s;
}

__device__ __forceinline__ float v2f_val(const DevGraph &G, const float *ev, const float *m,
                                         float bx, float mx, int vs, int es, int x) {
    return (mx == kNegInf) ? v2f_slow(G, ev, m, vs, es, x) : bx - mx;
}

// ---- log-sum-exp helpers -------------------------------------------------------------

// natural-log LSE of two values
__device__ __forceinline__ float lse2(float a, float b) {
    float mx = fmaxf(a, b), mn = fminf(a, b);
    if (mx == kNegInf || mx == pos_inf()) return mx;
    return mx + log1pf(expf(mn - mx));
}

// log(s(u)), s(u) = log(1 + e^u)
__device__ __forceinline__ float log_softplus(float u) {
    if (u < -15.f) return u + log1pf(-0.5f * expf(u));
    if (u > 0.f) return logf(u + log1pf(expf(-u)));
    return logf(log1pf(expf(u)));
}

// log(e^s - 1) from ls = log s
__device__ __forceinline__ float log_expm1_from_log(float ls) {
    if (ls == kNegInf) return kNegInf;
    if (ls == pos_inf()) return pos_inf();
    if (ls > 0.f) {
        float s = expf(ls);
        return s + logf(-expm1f(-s));
    }
    if (ls > -80.f) {
        float s = expf(ls);
        return ls + logf(expm1f(s) / s);
    }
    return ls;
}

// -log(1 - e^{-s}) from ls = log s
__device__ __forceinline__ float neg_log_1mexp_from_log(float ls) {
    if (ls == pos_inf()) return 0.f;
    if (ls > 0.f) return -logf(-expm1f(-expf(ls)));
    if (ls > -80.f) {
        float s = expf(ls);
        return -ls - logf(-expm1f(-s) / s);
    }
    return -ls;
}

// OR update to parent i (T > 0): ls = log of the leave-one-out softplus sum (in units
// of T), xc = child log-odds.
__device__ __forceinline__ float or_parent_soft(float ls, float xc, float T, float invT) {
    if (ls == kNegInf) return xc;
    float y = xc + T * log_expm1_from_log(ls);
    if (y >= 0.f) return T * neg_log_1mexp_from_log(ls) - T * log1pf(expf(-y * invT));
    return xc + T * expf(ls) - T * log1pf(expf(y * invT));
}

// OR update to parent i (T = 0): S = leave-one-out sum of max(x_j, 0), M = leave-one-out max.
__device__ __forceinline__ float or_parent_max(float S, float M, float xc) {
    float mn = M < 0.f ? M : 0.f;
    float z = xc + S + mn;
    return (z >= 0.f) ? -mn : xc + S;
}

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
        return mx + T * log1pf(expf((fminf(z[0], z[1]) - mx) * invT));
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

// Thread per variable. KFIX = 2: every variable binary (states at 2v, edge-states even).
template <int KFIX, int MODE>
__global__ void __launch_bounds__(256) k_var_thread(DevGraph G, const int32_t *__restrict__ list, int n,
                                                    const float *__restrict__ ev,
                                                    const float *__restrict__ m,
                                                    float *__restrict__ out,
                                                    int32_t *__restrict__ dec) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int v = list ? __ldg(list + t) : t;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    if constexpr (KFIX == 2) {
        const int vs = 2 * v;
        float2 s = __ldg(reinterpret_cast<const float2 *>(ev + vs));
        for (int k = k0; k < k1; ++k) {
            const int es = __ldg(G.vin_es + k);
            const float2 q = __ldg(reinterpret_cast<const float2 *>(m + es));
            s.x += q.x;
            s.y += q.y;
        }
        if constexpr (MODE == kVarBeliefs) {
            reinterpret_cast<float2 *>(out + vs)[0] = s;
        } else if constexpr (MODE == kVarNormalised) {
            float z = lse2(s.x, s.y);
            if (z == kNegInf) {
                atomicOr(G.flags, kFlagContradiction);
                reinterpret_cast<float2 *>(out + vs)[0] = make_float2(kNegInf, kNegInf);
            } else {
                if (s.x != s.x || s.y != s.y) atomicOr(G.flags, kFlagNaN);
                reinterpret_cast<float2 *>(out + vs)[0] = make_float2(s.x - z, s.y - z);
            }
        } else {
            dec[v] = (s.y > s.x) ? 1 : 0;
        }
    } else {
        const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
        float best = 0.f, mx = kNegInf;
        int arg = 0;
        bool nan = false;
        for (int x = 0; x < K; ++x) {
            float s = __ldg(ev + vs + x);
            for (int k = k0; k < k1; ++k) s += __ldg(m + __ldg(G.vin_es + k) + x);
            if constexpr (MODE == kVarBeliefs) out[vs + x] = s;
            if constexpr (MODE == kVarNormalised) {
                out[vs + x] = s;
                if (s > mx) mx = s;
                nan |= (s != s);
            }
            if constexpr (MODE == kVarDecode) {
                if (x == 0 || s > best) {
                    best = s;
                    arg = x;
                }
            }
        }
        if constexpr (MODE == kVarNormalised) {
            if (nan) atomicOr(G.flags, kFlagNaN);
            if (mx == kNegInf) {
                atomicOr(G.flags, kFlagContradiction);
            } else {
                float acc = 0.f;
                for (int x = 0; x < K; ++x) acc += expf(out[vs + x] - mx);
                const float z = mx + logf(acc);
                for (int x = 0; x < K; ++x) out[vs + x] -= z;
            }
        }
        if constexpr (MODE == kVarDecode) dec[v] = arg;
    }
}

// Block per (high-degree) variable; deterministic tree reduction.
template <int MODE>
__global__ void __launch_bounds__(256) k_var_block(DevGraph G, const int32_t *__restrict__ list,
                                                   const float *__restrict__ ev,
                                                   const float *__restrict__ m,
                                                   float *__restrict__ out,
                                                   int32_t *__restrict__ dec) {
    __shared__ float red[32];
    __shared__ float sb[kMaxStates];
    const int v = __ldg(list + blockIdx.x);
    const int vs = __ldg(G.vs_off + v), K = __ldg(G.vs_off + v + 1) - vs;
    const int k0 = __ldg(G.vin_off + v), k1 = __ldg(G.vin_off + v + 1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int x = 0; x < K; ++x) {
        float s = 0.f;
        for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) s += __ldg(m + __ldg(G.vin_es + k) + x);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.f;
            for (int w = 0; w < nw; ++w) tot += red[w];
            sb[x] = __ldg(ev + vs + x) + tot;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if constexpr (MODE == kVarBeliefs) {
        for (int x = 0; x < K; ++x) out[vs + x] = sb[x];
    } else if constexpr (MODE == kVarNormalised) {
        float mx = kNegInf;
        bool nan = false;
        for (int x = 0; x < K; ++x) {
            if (sb[x] > mx) mx = sb[x];
            nan |= (sb[x] != sb[x]);
        }
        if (nan) atomicOr(G.flags, kFlagNaN);
        if (mx == kNegInf) {
            atomicOr(G.flags, kFlagContradiction);
            for (int x = 0; x < K; ++x) out[vs + x] = kNegInf;
        } else {
            float acc = 0.f;
            for (int x = 0; x < K; ++x) acc += expf(sb[x] - mx);
            const float z = mx + logf(acc);
            for (int x = 0; x < K; ++x) out[vs + x] = sb[x] - z;
        }
    } else {
        int arg = 0;
        for (int x = 1; x < K; ++x)
            if (sb[x] > sb[arg]) arg = x;
        dec[v] = arg;
    }
}

// =====================================================================================
// Factor pass: dense pairwise tables (Ising, RBM, Potts), thread per factor
// =====================================================================================

template <int K, bool MAXP>
__global__ void __launch_bounds__(K >= 16 ? 128 : 256)
k_pair(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
       const float *__restrict__ b, const float *__restrict__ ev, const float *__restrict__ m_old,
       float *__restrict__ m_new, float T, float invT, float damping) {
    __shared__ float tab[K * K];
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int n_fac = __ldg(&S->n_fac), shared = __ldg(&S->shared), pot_base = __ldg(&S->pot_base);
    if (shared) {
        for (int i = threadIdx.x; i < K * K; i += blockDim.x) tab[i] = __ldg(pot + pot_base + i);
        __syncthreads();
    }
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= n_fac) return;
    const int e = __ldg(&S->edge_base) + 2 * f;
    const int es0 = __ldg(&S->es_base) + 2 * K * f, es1 = es0 + K;
    int vs0, vs1;
    if ((e & 1) == 0) {
        int2 q = __ldg(reinterpret_cast<const int2 *>(G.edge_vs + e));
        vs0 = q.x;
        vs1 = q.y;
    } else {
        vs0 = __ldg(G.edge_vs + e);
        vs1 = __ldg(G.edge_vs + e + 1);
    }
    float mo0[K], mo1[K], v0[K], v1[K];
    load_n_stream<K>(mo0, m_old + es0);
    load_n_stream<K>(mo1, m_old + es1);
    load_n<K>(v0, b + vs0);
    load_n<K>(v1, b + vs1);
#pragma unroll
    for (int x = 0; x < K; ++x) {
        v0[x] = v2f_val(G, ev, m_old, v0[x], mo0[x], vs0, es0, x);
        v1[x] = v2f_val(G, ev, m_old, v1[x], mo1[x], vs1, es1, x);
    }
    float o0[K], o1[K];
    if constexpr (K <= 4) {
        float phi[K * K];
        if (shared) {
#pragma unroll
            for (int i = 0; i < K * K; ++i) phi[i] = tab[i];
        } else {
            load_n<K * K>(phi, pot + pot_base + (size_t)f * (K * K));
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
        const float *phig = pot + pot_base + (size_t)f * (K * K);
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float z[K];
#pragma unroll
            for (int y = 0; y < K; ++y) z[y] = (shared ? tab[x * K + y] : __ldg(phig + x * K + y)) + v1[y];
            o0[x] = lse_row<K, MAXP>(z, T, invT);
        }
#pragma unroll
        for (int y = 0; y < K; ++y) {
            float z[K];
#pragma unroll
            for (int x = 0; x < K; ++x) z[x] = (shared ? tab[x * K + y] : __ldg(phig + x * K + y)) + v0[x];
            o1[y] = lse_row<K, MAXP>(z, T, invT);
        }
    }
    finish_k<K>(o0, mo0, damping, G.flags);
    finish_k<K>(o1, mo1, damping, G.flags);
    store_n<K>(m_new + es0, o0);
    store_n<K>(m_new + es1, o1);
}

// =====================================================================================
// Factor pass: any listed-configuration factor, thread per factor
// =====================================================================================

template <bool MAXP>
__global__ void __launch_bounds__(128)
k_enum_generic(DevGraph G, const EnumSeg *__restrict__ segs, int n_seg, const float *__restrict__ pot,
               const float *__restrict__ b, const float *__restrict__ ev,
               const float *__restrict__ m_old, float *__restrict__ m_new, float T, float invT,
               float damping) {
    const EnumSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
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
        for (int x = 0; x < Kj[j]; ++x) {
            const float mv = __ldg(m_old + es + x);
            mo[Ko[j] + x] = mv;
            v2f[Ko[j] + x] = v2f_val(G, ev, m_old, __ldg(b + vs + x), mv, vs, es, x);
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
    m_new[es] = t[0];
    m_new[es + 1] = t[1];
}

__device__ __forceinline__ float2 ld2(const float *p) { return make_float2(__ldg(p), __ldg(p + 1)); }

// Incoming log-odds of one edge (times sgn) and its stored message.
__device__ __forceinline__ float edge_logodds(const DevGraph &G, const float *ev, const float *b,
                                              const float *m_old, int e, int es, float sgn,
                                              float2 &mo) {
    const int vs = __ldg(G.edge_vs + e);
    mo = ld2(m_old + es);
    const float2 bb = ld2(b + vs);
    const float a0 = v2f_val(G, ev, m_old, bb.x, mo.x, vs, es, 0);
    const float a1 = v2f_val(G, ev, m_old, bb.y, mo.y, vs, es, 1);
    return sgn * log_odds(a0, a1);
}

// Thread per factor, fan-in <= kLogicSmallFan; leave-one-out sums written out directly.
template <bool MAXP>
__global__ void __launch_bounds__(256)
k_logic_small(DevGraph G, const LogicSeg *__restrict__ segs, int n_seg, const float *__restrict__ b,
              const float *__restrict__ ev, const float *__restrict__ m_old,
              float *__restrict__ m_new, float T, float invT, float damping) {
    const LogicSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * blockDim.x + threadIdx.x;
    if (f >= __ldg(&S->n_fac)) return;
    const int *po = G.paroff_pool + __ldg(&S->paroff_base);
    const int p0 = __ldg(po + f), n = __ldg(po + f + 1) - p0;
    const int edge_base = __ldg(&S->edge_base), es_base = __ldg(&S->es_base);
    const int e0 = edge_base + p0 + f;
    const float sgn = __ldg(&S->kind) == 1 ? -1.f : 1.f;
    float x[kLogicSmallFan + 1], u[kLogicSmallFan + 1];
    float2 mo[kLogicSmallFan + 1];
#pragma unroll
    for (int k = 0; k <= kLogicSmallFan; ++k) {
        if (k > n) break;
        const int e = e0 + k;
        x[k] = edge_logodds(G, ev, b, m_old, e, es_base + 2 * (e - edge_base), sgn, mo[k]);
    }
    const float xc = x[n];
    float out[kLogicSmallFan + 1];
    if (MAXP) {
        float A = 0.f, Mall = kNegInf;
        for (int j = 0; j < n; ++j) {
            A += fmaxf(x[j], 0.f);
            Mall = fmaxf(Mall, x[j]);
        }
        out[n] = A + (Mall < 0.f ? Mall : 0.f);
        for (int i = 0; i < n; ++i) {
            float Si = 0.f, Mi = kNegInf;
            for (int j = 0; j < n; ++j)
                if (j != i) {
                    Si += fmaxf(x[j], 0.f);
                    Mi = fmaxf(Mi, x[j]);
                }
            out[i] = or_parent_max(Si, Mi, xc);
        }
    } else {
        float Lall = kNegInf;
        for (int j = 0; j < n; ++j) {
            u[j] = log_softplus(x[j] * invT);
            Lall = lse2(Lall, u[j]);
        }
        out[n] = T * log_expm1_from_log(Lall);
        for (int i = 0; i < n; ++i) {
            float Li = kNegInf;
            for (int j = 0; j < n; ++j)
                if (j != i) Li = lse2(Li, u[j]);
            out[i] = or_parent_soft(Li, xc, T, invT);
        }
    }
    for (int k = 0; k <= n; ++k) {
        const int e = e0 + k;
        write_logic_edge(sgn * out[k], mo[k], m_new, es_base + 2 * (e - edge_base), damping, G.flags);
    }
}

// Combine operator of the warp scans: (+, max) for T = 0, (LSE, max) for T > 0.
template <bool MAXP>
__device__ __forceinline__ float comb(float a, float b) {
    if (MAXP) return a + b;
    return lse2(a, b);
}

// Warp per factor, any fan-in. Prefix and suffix leave-one-out sums by warp scans over
// rounds of 32 parents; per-parent values staged in shared memory (4 floats each).
template <bool MAXP>
__global__ void __launch_bounds__(128)
k_logic_warp(DevGraph G, const LogicSeg *__restrict__ segs, int n_seg, const float *__restrict__ b,
             const float *__restrict__ ev, const float *__restrict__ m_old,
             float *__restrict__ m_new, float T, float invT, float damping, int cap) {
    extern __shared__ float smem[];
    const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LogicSeg *S = segs + find_seg(segs, n_seg, blockIdx.x);
    const int f = (blockIdx.x - __ldg(&S->block_begin)) * warps + warp;
    if (f >= __ldg(&S->n_fac)) return;
    float *sx = smem + (size_t)warp * 4 * cap;  // x_j
    float *sv = sx + cap;                        // per-parent value (max(x,0) or log softplus)
    float *sp = sv + cap;                        // exclusive prefix of values
    float *sm = sp + cap;                        // exclusive prefix max of x
    const int *po = G.paroff_pool + __ldg(&S->paroff_base);
    const int p0 = __ldg(po + f), n = __ldg(po + f + 1) - p0;
    const int edge_base = __ldg(&S->edge_base), es_base = __ldg(&S->es_base);
    const int e0 = edge_base + p0 + f;
    const float sgn = __ldg(&S->kind) == 1 ? -1.f : 1.f;
    const float ident = MAXP ? 0.f : kNegInf;
    // child
    float2 moc = make_float2(0.f, 0.f);
    float xc = 0.f;
    if (lane == 0) xc = edge_logodds(G, ev, b, m_old, e0 + n, es_base + 2 * (e0 + n - edge_base), sgn, moc);
    xc = __shfl_sync(0xffffffffu, xc, 0);
    // forward pass: exclusive prefix
    float ca = ident, cm = kNegInf;
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        const bool valid = j < n;
        float xv = 0.f, va = ident, vm = kNegInf;
        if (valid) {
            float2 mo;
            const int e = e0 + j;
            xv = edge_logodds(G, ev, b, m_old, e, es_base + 2 * (e - edge_base), sgn, mo);
            va = MAXP ? fmaxf(xv, 0.f) : log_softplus(xv * invT);
            vm = xv;
        }
        float ia = va, im = vm;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float ya = __shfl_up_sync(0xffffffffu, ia, d);
            const float ym = __shfl_up_sync(0xffffffffu, im, d);
            if (lane >= d) {
                ia = comb<MAXP>(ya, ia);
                im = fmaxf(ym, im);
            }
        }
        float ea = __shfl_up_sync(0xffffffffu, ia, 1), em = __shfl_up_sync(0xffffffffu, im, 1);
        if (lane == 0) {
            ea = ident;
            em = kNegInf;
        }
        if (valid) {
            sx[j] = xv;
            sv[j] = va;
            sp[j] = comb<MAXP>(ca, ea);
            sm[j] = fmaxf(cm, em);
        }
        ca = comb<MAXP>(ca, __shfl_sync(0xffffffffu, ia, 31));
        cm = fmaxf(cm, __shfl_sync(0xffffffffu, im, 31));
    }
    __syncwarp();
    const float out_c = MAXP ? ca + (cm < 0.f ? cm : 0.f) : T * log_expm1_from_log(ca);
    // backward pass: exclusive suffix, outputs
    float sa = ident, smx = kNegInf;
    for (int base = n > 0 ? ((n - 1) & ~31) : -32; base >= 0; base -= 32) {
        const int j = base + lane;
        const bool valid = j < n;
        const float va = valid ? sv[j] : ident;
        const float vm = valid ? sx[j] : kNegInf;
        float ra = va, rm = vm;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float ya = __shfl_down_sync(0xffffffffu, ra, d);
            const float ym = __shfl_down_sync(0xffffffffu, rm, d);
            if (lane + d < 32) {
                ra = comb<MAXP>(ra, ya);
                rm = fmaxf(rm, ym);
            }
        }
        float ea = __shfl_down_sync(0xffffffffu, ra, 1), em = __shfl_down_sync(0xffffffffu, rm, 1);
        if (lane == 31) {
            ea = ident;
            em = kNegInf;
        }
        ea = comb<MAXP>(ea, sa);
        em = fmaxf(em, smx);
        if (valid) {
            const float loo_a = comb<MAXP>(sp[j], ea);
            const float loo_m = fmaxf(sm[j], em);
            const float o = MAXP ? or_parent_max(loo_a, loo_m, xc) : or_parent_soft(loo_a, xc, T, invT);
            const int e = e0 + j;
            const int es = es_base + 2 * (e - edge_base);
            write_logic_edge(sgn * o, ld2(m_old + es), m_new, es, damping, G.flags);
        }
        sa = comb<MAXP>(sa, __shfl_sync(0xffffffffu, ra, 0));
        smx = fmaxf(smx, __shfl_sync(0xffffffffu, rm, 0));
    }
    if (lane == 0) {
        const int e = e0 + n;
        write_logic_edge(sgn * out_c, moc, m_new, es_base + 2 * (e - edge_base), damping, G.flags);
    }
}

}  // namespace

// =====================================================================================
// Launchers
// =====================================================================================

cudaError_t prepare_kernels(int max_smem_bytes) {
    cudaError_t e = cudaSuccess;
    if (max_smem_bytes > 48 * 1024) {
        e = cudaFuncSetAttribute(k_logic_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_logic_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
    }
    return e;
}

template <int MODE>
static void var_pass_mode(const DevGraph &G, const Plan &P, const float *ev, const float *m,
                          float *out, int32_t *dec, cudaStream_t s) {
    for (const VarLaunch &L : P.var) {
        if (L.n == 0) continue;
        if (L.block_mode) {
            k_var_block<MODE><<<L.n, L.threads, 0, s>>>(G, L.list, ev, m, out, dec);
        } else if (P.kfix == 2) {
            k_var_thread<2, MODE><<<L.n_blocks, L.threads, 0, s>>>(G, L.list, L.n, ev, m, out, dec);
        } else {
            k_var_thread<0, MODE><<<L.n_blocks, L.threads, 0, s>>>(G, L.list, L.n, ev, m, out, dec);
        }
    }
}

cudaError_t launch_var_pass(const DevGraph &G, const Plan &P, const float *ev, const float *m,
                            float *b, int mode, int32_t *decode, cudaStream_t s) {
    if (mode == kVarBeliefs) var_pass_mode<kVarBeliefs>(G, P, ev, m, b, decode, s);
    else if (mode == kVarNormalised) var_pass_mode<kVarNormalised>(G, P, ev, m, b, decode, s);
    else var_pass_mode<kVarDecode>(G, P, ev, m, b, decode, s);
    return cudaGetLastError();
}

template <bool MAXP>
static void factor_pass_t(const DevGraph &G, const Plan &P, const float *pot, const float *b,
                          const float *ev, const float *m_old, float *m_new, float T, float damping,
                          cudaStream_t s) {
    const float invT = MAXP ? 0.f : 1.f / T;
    for (const FactorLaunch &L : P.factor) {
        if (L.n_blocks == 0) continue;
        const EnumSeg *es = static_cast<const EnumSeg *>(L.segs);
        const LogicSeg *ls = static_cast<const LogicSeg *>(L.segs);
        switch (L.variant) {
            case kPair2:
                k_pair<2, MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair4:
                k_pair<4, MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair8:
                k_pair<8, MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kPair16:
                k_pair<16, MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kEnumGeneric:
                k_enum_generic<MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, es, L.n_seg, pot, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kLogicSmall:
                k_logic_small<MAXP><<<L.n_blocks, L.threads, 0, s>>>(G, ls, L.n_seg, b, ev, m_old, m_new, T, invT, damping);
                break;
            case kLogicWarp:
                k_logic_warp<MAXP><<<L.n_blocks, L.threads, L.smem, s>>>(G, ls, L.n_seg, b, ev, m_old, m_new, T, invT, damping, L.max_fan);
                break;
            default:
                break;
        }
    }
}

cudaError_t launch_factor_pass(const DevGraph &G, const Plan &P, const float *log_pot,
                               const float *b, const float *ev, const float *m_old,
                               float *m_new, float T, float damping, cudaStream_t s) {
    if (T == 0.f) factor_pass_t<true>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s);
    else factor_pass_t<false>(G, P, log_pot, b, ev, m_old, m_new, T, damping, s);
    return cudaGetLastError();
}

}  // namespace pgm
