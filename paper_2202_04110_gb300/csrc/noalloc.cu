// Allocation-free LBP on 4-neighbour grids of binary variables (pgm_grid2_run_bp_noalloc).
//
// For callers that cannot allocate device memory: pgm_build and pgm_run_bp need device
// memory for the compiled index arrays and the per-graph scratch, which a process
// whose device memory is owned and budgeted by a host framework (or which must not
// call cudaMalloc / cudaFree after start-up) cannot obtain. This entry point needs no
// graph object: the grid topology is computed from (row, column), and the scratch --
// the ping-pong partner of the caller's message buffer, the per-iteration beliefs and a
// status word -- lives in one file-scope static __device__ array of fixed size. Every
// GPU that loads the library holds that array until the process exits.
//
// It computes the same iteration as pgm_run_bp on the graph that pgm_build makes from a
// grid whose factors are listed cell by cell (right pair, then down pair), with the same
// message layout, so the two can be compared directly.
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>
#include <math_constants.h>

#include "../../include/pgm.h"
#include "pgm_internal.h"

namespace {

constexpr int kStatusFloats = 64;  // a 256-byte slot for the status word
constexpr int64_t kScratchFloats = PGM_NOALLOC_SCRATCH_FLOATS;

// The whole scratch: [status slot | message buffer (ES) | beliefs (VS)]. Host code must
// never pass this symbol to a kernel (on the host it is only a stand-in); it uses the
// device address from cudaGetSymbolAddress instead.
static __device__ __align__(256) float g_noalloc_scratch[kStatusFloats + kScratchFloats];

constexpr float kExact = 128.f;

__device__ __forceinline__ float ninf() { return -CUDART_INF_F; }

// first factor of cell (r, c): cells of non-last rows own a right and a down factor
// (the last column only a down one), the last row only right factors
__device__ __forceinline__ int fbase(int r, int c, int rows, int cols) {
    return r * (2 * cols - 1) + c * (r < rows - 1 ? 2 : 1);
}

// incoming edge-states of variable (r, c), in ascending edge order
__device__ __forceinline__ int grid_in_es(int r, int c, int rows, int cols, int (&es)[4]) {
    int n = 0;
    if (r > 0) es[n++] = 4 * (fbase(r - 1, c, rows, cols) + (c < cols - 1 ? 1 : 0)) + 2;
    if (c > 0) es[n++] = 4 * fbase(r, c - 1, rows, cols) + 2;
    if (c < cols - 1) es[n++] = 4 * fbase(r, c, rows, cols);
    if (r < rows - 1) es[n++] = 4 * (fbase(r, c, rows, cols) + (c < cols - 1 ? 1 : 0));
    return n;
}

// the two variables of factor f
__device__ __forceinline__ void grid_factor_vars(int f, int rows, int cols, int &v0, int &v1) {
    const int per_row = 2 * cols - 1;
    const int full = (rows - 1) * per_row;
    if (f < full) {
        const int r = f / per_row, q = f - r * per_row, c = q >> 1;
        v0 = r * cols + c;
        v1 = ((q & 1) == 0 && c < cols - 1) ? v0 + 1 : v0 + cols;
    } else {
        v0 = (rows - 1) * cols + (f - full);
        v1 = v0 + 1;
    }
}

// compensated sum s + v (hi, lo)
__device__ __forceinline__ void two_sum(float &hi, float &lo, float v) {
    const float s = hi + v;
    if (!isfinite(s)) {
        hi = s;
        lo = 0.f;
        return;
    }
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

__device__ __forceinline__ float ff_rel(float ahi, float alo, float bhi, float blo) {
    if (!isfinite(ahi) || !isfinite(bhi)) return ahi - bhi;
    return (ahi - bhi) + (alo - blo);
}

// beliefs of variable (r, c) relative to its larger state, from e + sum of incoming
// messages except edge-state `skip` (-1: none)
__device__ __forceinline__ float2 grid_sum(int r, int c, int rows, int cols, const float *ev,
                                           const float *m, int skip, bool relative) {
    int es[4];
    const int n = grid_in_es(r, c, rows, cols, es);
    const int v = r * cols + c;
    float h0 = ev[2 * v], l0 = 0.f, h1 = ev[2 * v + 1], l1 = 0.f;
    for (int k = 0; k < n; ++k) {
        if (es[k] == skip) continue;
        const float2 q = *reinterpret_cast<const float2 *>(m + es[k]);
        two_sum(h0, l0, q.x);
        two_sum(h1, l1, q.y);
    }
    if (!relative) return make_float2(h0 + l0, h1 + l1);
    if (h0 == ninf() && h1 == ninf()) return make_float2(ninf(), ninf());
    const float d = ff_rel(h1, l1, h0, l0);
    return d > 0.f ? make_float2(ff_rel(h0, l0, h1, l1), 0.f) : make_float2(0.f, d);
}

__global__ void __launch_bounds__(256) k_grid_var(int rows, int cols, const float *__restrict__ ev,
                                                  const float *__restrict__ m, float *__restrict__ b) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= rows * cols) return;
    const int r = v / cols, c = v - r * cols;
    reinterpret_cast<float2 *>(b)[v] = grid_sum(r, c, rows, cols, ev, m, -1, true);
}

template <bool MAXP>
__device__ __forceinline__ float lse_pair(float a, float b, float T, float invT) {
    const float mx = fmaxf(a, b);
    if (MAXP || mx == ninf()) return mx;
    return mx + T * log1pf(expf((fminf(a, b) - mx) * invT));
}

__device__ __forceinline__ void norm2(float &a, float &b, unsigned *status) {
    const float mx = fmaxf(a, b);
    if (mx == ninf()) {  // a contradiction: the message becomes 0 and the status records it
        a = b = 0.f;
        atomicOr(status, PGM_FLAG_CONTRADICTION);
        return;
    }
    a -= mx;
    b -= mx;
}

template <bool MAXP>
__global__ void __launch_bounds__(256) k_grid_pair(int rows, int cols, int n_fac, const float *__restrict__ pot,
                                                   const float *__restrict__ ev, const float *__restrict__ b,
                                                   const float *__restrict__ m_old, float *__restrict__ m_new,
                                                   float T, float invT, float damping, unsigned *status) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_fac) return;
    int v0, v1;
    grid_factor_vars(f, rows, cols, v0, v1);
    const float4 mo = *reinterpret_cast<const float4 *>(m_old + 4 * f);
    const float4 phi = *reinterpret_cast<const float4 *>(pot + 4 * f);
    float2 a, c;  // variable-to-factor values of edge 0 (v0) and edge 1 (v1)
    if (!(fabsf(mo.x) <= kExact && fabsf(mo.y) <= kExact)) {
        a = grid_sum(v0 / cols, v0 % cols, rows, cols, ev, m_old, 4 * f, false);
    } else {
        const float2 bb = reinterpret_cast<const float2 *>(b)[v0];
        a = make_float2(bb.x - mo.x, bb.y - mo.y);
    }
    if (!(fabsf(mo.z) <= kExact && fabsf(mo.w) <= kExact)) {
        c = grid_sum(v1 / cols, v1 % cols, rows, cols, ev, m_old, 4 * f + 2, false);
    } else {
        const float2 bb = reinterpret_cast<const float2 *>(b)[v1];
        c = make_float2(bb.x - mo.z, bb.y - mo.w);
    }
    // to v0: LSE over v1's state; to v1: LSE over v0's state (configurations 00,01,10,11)
    float o0 = lse_pair<MAXP>(phi.x + c.x, phi.y + c.y, T, invT);
    float o1 = lse_pair<MAXP>(phi.z + c.x, phi.w + c.y, T, invT);
    float p0 = lse_pair<MAXP>(phi.x + a.x, phi.z + a.y, T, invT);
    float p1 = lse_pair<MAXP>(phi.y + a.x, phi.w + a.y, T, invT);
    norm2(o0, o1, status);
    norm2(p0, p1, status);
    if (damping != 0.f) {
        const float w = 1.f - damping;
        o0 = damping * mo.x + w * o0;
        o1 = damping * mo.y + w * o1;
        p0 = damping * mo.z + w * p0;
        p1 = damping * mo.w + w * p1;
    }
    norm2(o0, o1, status);
    norm2(p0, p1, status);
    *reinterpret_cast<float4 *>(m_new + 4 * f) = make_float4(o0, o1, p0, p1);
}

std::mutex g_setup_mu;
float *g_scratch_ptr[64] = {};

// Once per device, with that device current: the device address of the static array.
cudaError_t scratch_for_current_device(float **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pgm_status pgm_grid2_run_bp_noalloc(int32_t rows, int32_t cols, const float *log_pot,
                                               const float *evidence, float T, float damping,
                                               int32_t n_iters, float *msgs, void *stream) {
    if (rows < 1 || cols < 1) return pgm::set_last_error(PGM_EINVAL, "rows and cols must be >= 1");
    const int64_t V = (int64_t)rows * cols;
    const int64_t F = (int64_t)rows * (cols - 1) + (int64_t)(rows - 1) * cols;
    const int64_t ES = 4 * F, VS = 2 * V;
    if (ES + VS > kScratchFloats)
        return pgm::set_last_error(
            PGM_EINVAL, "grid " + std::to_string(rows) + "x" + std::to_string(cols) + " needs " +
                            std::to_string(ES + VS) + " floats of scratch; the allocation-free path has " +
                            std::to_string(kScratchFloats) + " (4 * factors + 2 * variables must fit)");
    if (!(T >= 0.f) || !std::isfinite(T)) return pgm::set_last_error(PGM_EINVAL, "T must be finite and >= 0");
    if (!(damping >= 0.f && damping < 1.f)) return pgm::set_last_error(PGM_EINVAL, "damping must be in [0, 1)");
    if (n_iters < 0) return pgm::set_last_error(PGM_EINVAL, "n_iters must be >= 0");
    if (!evidence || (F > 0 && (!log_pot || !msgs))) return pgm::set_last_error(PGM_EINVAL, "NULL argument");
    if ((reinterpret_cast<uintptr_t>(log_pot) | reinterpret_cast<uintptr_t>(msgs)) & 15u ||
        reinterpret_cast<uintptr_t>(evidence) & 7u)
        return pgm::set_last_error(PGM_EINVAL, "log_pot and msgs must be 16-byte aligned, evidence 8-byte aligned");
    if (n_iters == 0 || F == 0) return PGM_OK;
    float *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess)
        return pgm::set_last_error(PGM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned *status = reinterpret_cast<unsigned *>(scratch);
    float *m_tmp = scratch + kStatusFloats;
    float *b = m_tmp + ES;
    // the status word is the only scratch that must start at zero (it then holds this
    // call's PGM_FLAG_* bits, read with pgm_grid2_noalloc_flags); the message buffer and
    // the beliefs are fully written before they are read
    e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const float invT = T > 0.f ? 1.f / T : 0.f;
    const int vb = (int)((V + 255) / 256), fb = (int)((F + 255) / 256);
    float *cur = msgs, *nxt = m_tmp;
    for (int it = 0; it < n_iters; ++it) {
        k_grid_var<<<vb, 256, 0, s>>>(rows, cols, evidence, cur, b);
        if (T == 0.f)
            k_grid_pair<true><<<fb, 256, 0, s>>>(rows, cols, (int)F, log_pot, evidence, b, cur, nxt, T, invT, damping, status);
        else
            k_grid_pair<false><<<fb, 256, 0, s>>>(rows, cols, (int)F, log_pot, evidence, b, cur, nxt, T, invT, damping, status);
        float *t = cur;
        cur = nxt;
        nxt = t;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (cur != msgs) {
        e = cudaMemcpyAsync(msgs, cur, (size_t)ES * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    }
    return PGM_OK;
}

extern "C" pgm_status pgm_grid2_noalloc_flags(uint32_t *flags, int32_t clear, void *stream) {
    if (!flags) return pgm::set_last_error(PGM_EINVAL, "flags is NULL");
    float *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess)
        return pgm::set_last_error(PGM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e));
    e = cudaMemcpy(flags, scratch, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    if (clear) {
        e = cudaMemset(scratch, 0, sizeof(uint32_t));
        if (e != cudaSuccess) return pgm::set_last_error(PGM_ECUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    }
    return PGM_OK;
}
