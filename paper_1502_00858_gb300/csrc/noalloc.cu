// calib_eval_noalloc: the residual/gradient evaluation of calib_eval for callers that cannot
// allocate device memory. It takes every input and output from the caller and keeps its only
// scratch - per-chunk partial station sums - in a fixed array in this file's device memory.
//
// Who needs it: applications whose device memory is entirely reserved by their own pool
// allocator (a cudaMalloc would fail or fragment that pool), and latency-critical pipelines that
// cannot afford the implicit device synchronisation of cudaMalloc / cudaFree.
//
// Scratch rules: the array is shared by every call in the process on a given device and keeps
// the previous call's contents; each call overwrites every slot it later reads, so nothing needs
// clearing. Calls that overlap on the GPU (different streams, or other threads) race on it.
// The station sums are accumulated with shared-memory atomics, so the result is not bitwise
// reproducible from call to call (it varies in the last bits; calib_eval is reproducible).
// Station pairs are validated on the device: a pair outside 0 <= p < q < N is skipped, and its
// chunk marks the agent's results invalid (L, g and grad are written as NaN).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "calib.h"
#include "calib_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;         // 4 threads per baseline, 64 baselines per pass
constexpr int NA_BASELINES_PER_CTA = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[CALIB_NOALLOC_SCRATCH_BYTES];

struct NoAllocArgs {
    const float2* vis;   // [A][B][T][4]
    const float2* coh;   // [A][B][T][K]
    const int* pq;       // [B][2]
    const float* J;      // [A][K][N][8]
    const float* Y;      // [A][K][N][8] or null
    const float* BZ;     // [A][K][N][8] or null
    float rho[16];
    float* part;         // scratch: [A][n_chunks][K][N][8]
    double* part_cost;   // scratch: [A][n_chunks]
    double* L;           // [A]
    double* g;           // [A]
    float* grad;         // [A][K][N][8]
    int A, N, B, K, T, n_chunks;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmul_cb(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
__device__ __forceinline__ float2 cmul_ca(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// One CTA per (chunk of NA_BASELINES_PER_CTA baselines, agent); four threads per baseline, one per
// correlation. R_t = V_t - sum_k c_tk J_pk J_qk^H; station p gets -sum_t conj(c_tk) R_t J_qk and
// station q gets -sum_t c_tk R_t^H J_pk, summed in shared memory, written to the scratch slot.
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_sweep(const NoAllocArgs a) {
    extern __shared__ __align__(16) float2 sm[];
    const int agent = blockIdx.y, chunk = blockIdx.x;
    const int N = a.N, K = a.K, KN4 = K * N * 4;
    float2* Js = sm;          // [K][N][4]
    float2* acc = sm + KN4;   // [K][N][4]
    __shared__ double red[32];
    const int tid = threadIdx.x, lane = tid & 31, gbase = lane & ~3, e = tid & 3, rr = e >> 1, cc = e & 1;
    const float2* Jg = reinterpret_cast<const float2*>(a.J) + (size_t)agent * KN4;
    for (int i = tid; i < KN4; i += blockDim.x) {
        Js[i] = Jg[i];
        acc[i] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    double cost = 0.0;
    bool bad = false;  // this thread met a station pair outside 0 <= p < q < N
    const int b_begin = chunk * NA_BASELINES_PER_CTA;
    const int b_end = min(a.B, b_begin + NA_BASELINES_PER_CTA);
    for (int b0 = b_begin; b0 < b_end; b0 += NA_THREADS / 4) {
        const int b = b0 + (tid >> 2);
        int p = 0, q = 0;
        bool active = b < b_end;
        if (active) {
            p = a.pq[2 * b];
            q = a.pq[2 * b + 1];
            if (!(p >= 0 && p < q && q < N)) {  // never index shared memory with a bad pair
                bad = true;
                active = false;
                p = q = 0;
            }
        }
        float2 P[16], W[16];
        for (int k = 0; k < K; ++k) {
            const float2* jp = Js + (k * N + p) * 4;
            const float2* jq = Js + (k * N + q) * 4;
            P[k] = add2(cmul_cb(jp[rr * 2 + 0], jq[cc * 2 + 0]), cmul_cb(jp[rr * 2 + 1], jq[cc * 2 + 1]));
            W[k] = make_float2(0.f, 0.f);
        }
        if (active) {
            for (int t = 0; t < a.T; ++t) {
                const size_t vis_i = ((size_t)agent * a.B + b) * a.T + t;
                const float2* cp = a.coh + vis_i * K;
                float2 m = make_float2(0.f, 0.f);
                for (int k = 0; k < K; ++k) m = add2(m, cmul(cp[k], P[k]));
                const float2 v = a.vis[vis_i * 4 + e];
                const float2 r = make_float2(v.x - m.x, v.y - m.y);
                cost += (double)r.x * r.x + (double)r.y * r.y;
                for (int k = 0; k < K; ++k) W[k] = add2(W[k], cmul_ca(cp[k], r));
            }
        }
        for (int k = 0; k < K; ++k) {
            // all lanes take part in the shuffles; inactive baselines carry W = 0
            const float2 w_r0 = shfl2(W[k], gbase + rr * 2 + 0), w_r1 = shfl2(W[k], gbase + rr * 2 + 1);
            const float2 w_0r = shfl2(W[k], gbase + 0 * 2 + rr), w_1r = shfl2(W[k], gbase + 1 * 2 + rr);
            if (active) {
                const float2* jq = Js + (k * N + q) * 4;
                const float2* jp = Js + (k * N + p) * 4;
                const float2 to_p = add2(cmul(w_r0, jq[0 * 2 + cc]), cmul(w_r1, jq[1 * 2 + cc]));
                const float2 to_q = add2(cmul_ca(w_0r, jp[0 * 2 + cc]), cmul_ca(w_1r, jp[1 * 2 + cc]));
                float* dp = reinterpret_cast<float*>(acc + (k * N + p) * 4 + e);
                float* dq = reinterpret_cast<float*>(acc + (k * N + q) * 4 + e);
                atomicAdd(dp, -to_p.x);
                atomicAdd(dp + 1, -to_p.y);
                atomicAdd(dq, -to_q.x);
                atomicAdd(dq + 1, -to_q.y);
            }
        }
    }
    __syncthreads();
    float2* out = reinterpret_cast<float2*>(a.part) + ((size_t)agent * a.n_chunks + chunk) * KN4;
    for (int i = tid; i < KN4; i += blockDim.x) out[i] = acc[i];
    const bool any_bad = __syncthreads_or(bad);
    for (int o = 16; o > 0; o >>= 1) cost += __shfl_down_sync(0xffffffffu, cost, o);
    if (lane == 0) red[tid >> 5] = cost;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        // a NaN cost is the chunk's "invalid pair" mark (read by k_noalloc_finish)
        a.part_cost[(size_t)agent * a.n_chunks + chunk] = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : s;
    }
}

// Per agent: grad = sum of the chunk partials + Y/2 + rho/2 (J - BZ) (Eq. gradL); g and
// L = g + Re tr(Y^H D) + rho/2 ||D||^2 (Eq. sumtrace2).
__global__ void __launch_bounds__(NA_THREADS) k_noalloc_finish(const NoAllocArgs a) {
    __shared__ double red[33];
    const int agent = blockIdx.x;
    const int KN8 = a.K * a.N * 8;
    bool bad = false;  // a chunk of this agent met an invalid station pair
    for (int ch = 0; ch < a.n_chunks; ++ch) bad = bad || isnan(a.part_cost[(size_t)agent * a.n_chunks + ch]);
    const float fnan = __int_as_float(0x7fc00000);
    double pen = 0.0;
    for (int i = threadIdx.x; i < KN8; i += blockDim.x) {
        const size_t o = (size_t)agent * KN8 + i;
        const double rk = a.rho[i / (a.N * 8)];
        float s = 0.f;
        for (int ch = 0; ch < a.n_chunks; ++ch) s += a.part[((size_t)agent * a.n_chunks + ch) * KN8 + i];
        const double y = a.Y ? (double)a.Y[o] : 0.0;
        const double d = (double)a.J[o] - (a.BZ ? (double)a.BZ[o] : 0.0);
        a.grad[o] = bad ? fnan : (float)((double)s + 0.5 * y + 0.5 * rk * d);
        pen += y * d + 0.5 * rk * d * d;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) pen += __shfl_down_sync(0xffffffffu, pen, o);
    if (lane == 0) red[w] = pen;
    __syncthreads();
    if (threadIdx.x == 0) {
        double p = 0.0, g = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) p += red[i];
        for (int ch = 0; ch < a.n_chunks; ++ch) g += a.part_cost[(size_t)agent * a.n_chunks + ch];
        if (bad) g = p = __longlong_as_double(0x7ff8000000000000LL);
        if (a.g) a.g[agent] = g;
        if (a.L) a.L[agent] = g + p;
    }
}

std::mutex g_na_mutex;
void* g_na_scratch_ptr[64] = {nullptr};

int na_fail(int code, const std::string& m) {
    calib::set_last_error(m);
    return code;
}

}  // namespace

extern "C" int calib_eval_noalloc(int n_agents, int n_stations, int n_baselines, int n_dirs, int n_samples,
                                  const int32_t* pq, const void* vis, const void* coh, const void* J,
                                  const void* Y, const void* BZ, const double* rho, double* L, double* g,
                                  void* grad, void* cuda_stream) {
    const int A = n_agents, N = n_stations, B = n_baselines, K = n_dirs, T = n_samples;
    if (A < 1 || N < 2 || N > 128 || B < 1 || K < 1 || K > 16 || T < 1)
        return na_fail(CALIB_EINVAL, "calib_eval_noalloc: sizes out of range (N in [2,128], K in [1,16])");
    if (!pq || !vis || !coh || !J || !rho || !grad)
        return na_fail(CALIB_EINVAL, "calib_eval_noalloc: pq, vis, coh, J, rho and grad are required");
    for (int k = 0; k < K; ++k)
        if (!(rho[k] > 0.0)) return na_fail(CALIB_EINVAL, "calib_eval_noalloc: rho must be > 0");
    const int n_chunks = (B + NA_BASELINES_PER_CTA - 1) / NA_BASELINES_PER_CTA;
    const size_t part_bytes = (size_t)A * n_chunks * K * N * 8 * sizeof(float);
    const size_t cost_bytes = (size_t)A * n_chunks * sizeof(double);
    const size_t cost_off = (part_bytes + 255) / 256 * 256;
    if (cost_off + cost_bytes > (size_t)CALIB_NOALLOC_SCRATCH_BYTES)
        return na_fail(CALIB_EINVAL, "calib_eval_noalloc: problem needs " + std::to_string(cost_off + cost_bytes) +
                                         " bytes of scratch, more than the fixed " +
                                         std::to_string((long long)CALIB_NOALLOC_SCRATCH_BYTES));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return na_fail(CALIB_ECUDA, "calib_eval_noalloc: no usable current device");
    void* scratch = nullptr;
    {
        // First call on a device: look up the device address of the scratch array once, with that
        // device current (the host-side name is only a stand-in for it).
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return na_fail(CALIB_ECUDA, std::string("calib_eval_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_scratch_ptr[dev] = p;
        }
        scratch = g_na_scratch_ptr[dev];
    }
    NoAllocArgs a{};
    a.vis = static_cast<const float2*>(vis);
    a.coh = static_cast<const float2*>(coh);
    a.pq = pq;
    a.J = static_cast<const float*>(J);
    a.Y = static_cast<const float*>(Y);
    a.BZ = static_cast<const float*>(BZ);
    for (int k = 0; k < K; ++k) a.rho[k] = (float)rho[k];
    a.part = static_cast<float*>(scratch);
    a.part_cost = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + cost_off);
    a.L = L;
    a.g = g;
    a.grad = static_cast<float*>(grad);
    a.A = A; a.N = N; a.B = B; a.K = K; a.T = T; a.n_chunks = n_chunks;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t smem = (size_t)2 * K * N * 4 * sizeof(float2);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_noalloc_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return na_fail(CALIB_ECUDA, std::string("calib_eval_noalloc: ") + cudaGetErrorString(e));
    }
    k_noalloc_sweep<<<dim3(n_chunks, A), NA_THREADS, smem, s>>>(a);
    k_noalloc_finish<<<A, NA_THREADS, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(CALIB_ECUDA, std::string("calib_eval_noalloc: launch: ") + cudaGetErrorString(e));
    return CALIB_OK;
}
