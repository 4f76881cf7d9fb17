// Learned warm start of the J-update: a small multilayer perceptron trained on solutions the
// C-ADMM itself produced (the paper starts each calibration from the previous time slot's
// solution, Section 3, initialisation; the network refines that start).
//
// Rows: one per (agent, direction, station): x = [J_prev (8 reals), (B_f Z_prev) (8 reals),
// normalised frequency]; the network outputs a correction y and J_init = J_prev + y.
// Dense layers with ReLU between them; bfloat16 weights and biases (copies of float32 master
// weights), float32 activations and accumulation; mean squared error; AdamW. Every reduction has
// a fixed order. The GEMMs run on the tensor cores (mma.sync TF32 with a hi/lo split of the float32
// operands, float32 accumulation), tiled 64x64x16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "calib.h"
#include "calib_internal.cuh"

namespace calib {
namespace {

enum Epi : int { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2, EPI_MASK = 3 };

__device__ __forceinline__ float ldf(const float* p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[M][N] = op(A)[M][K] op(B)[K][N] with an epilogue; A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n].
//
// Tensor cores: warp-level mma.sync m16n8k8 with TF32 operands and float32 accumulation. A TF32
// value keeps 10 mantissa bits, so a float32 operand x is split into hi = tf32(x) and
// lo = tf32(x - hi) (x - hi is exact in float32 and lo carries its next 11 bits), and a product is
// the sum of the partial products hi*hi + hi*lo + lo*hi (the lo*lo term is below float32 round-off;
// Henry, Tang and Heinecke 2019 use the same three-product split for bfloat16). bfloat16 values
// (the weights) are exact in TF32 and need no lo part, so a bfloat16 operand costs two products.
// CTA tile 64 x 64, k-step 16, 4 warps in a 2 x 2 grid of 32 x 32 warp tiles (2 x 4 mma tiles).
// Operands are staged in shared memory as float32, rows padded to 20 floats: the fragment reads
// (8 rows x 4 columns a warp) then fall on 32 distinct banks.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename T> struct IsBf16 { static constexpr bool value = false; };
template <> struct IsBf16<__nv_bfloat16> { static constexpr bool value = true; };

constexpr int GT_M = 64, GT_N = 64, GT_K = 16, GT_LD = GT_K + 4;
constexpr int SPLITK_MAX = 16;  // K-splits of a weight-gradient product

template <typename TAE, typename TBE, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const TAE* __restrict__ A, int lda,
                                              const TBE* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const __nv_bfloat16* __restrict__ bias, const float* __restrict__ mask,
                                              int ldm, int k_chunk) {
    constexpr bool A_EXACT = IsBf16<TAE>::value, B_EXACT = IsBf16<TBE>::value;
    constexpr int PER = GT_M * GT_K / 128;  // tile elements a thread stages per operand
    __shared__ float As[GT_M][GT_LD];  // As[m][k]
    __shared__ float Bs[GT_N][GT_LD];  // Bs[n][k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * GT_M, n0 = blockIdx.x * GT_N;
    // split-K: this CTA sums k in [kb, ke) and writes its partial to C + blockIdx.z * M * ldc
    const int kb = blockIdx.z * k_chunk, ke = min(K, kb + k_chunk);
    float* Cz = C + (size_t)blockIdx.z * M * ldc;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    // staging map: consecutive threads take consecutive elements of the index contiguous in memory
    auto a_at = [](int e, int& mm, int& kk) {
        kk = TA ? e / GT_M : e % GT_K;
        mm = TA ? e % GT_M : e / GT_K;
    };
    auto b_at = [](int e, int& nn, int& kk) {
        kk = TB ? e % GT_K : e / GT_N;
        nn = TB ? e / GT_K : e % GT_N;
    };
    float ra[PER], rb[PER];  // the next k-tile, fetched while the current one is multiplied
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = threadIdx.x + q * 128;
            int mm, kk, nn, kq;
            a_at(e, mm, kk);
            const int m = m0 + mm, k = k0 + kk;
            ra[q] = (m < M && k < ke) ? ldf(TA ? A + (size_t)k * lda + m : A + (size_t)m * lda + k) : 0.f;
            b_at(e, nn, kq);
            const int n = n0 + nn, k2 = k0 + kq;
            rb[q] = (n < N && k2 < ke) ? ldf(TB ? B + (size_t)n * ldb + k2 : B + (size_t)k2 * ldb + n) : 0.f;
        }
    };
    auto stage = [&]() {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int e = threadIdx.x + q * 128;
            int mm, kk, nn, kq;
            a_at(e, mm, kk);
            As[mm][kk] = ra[q];
            b_at(e, nn, kq);
            Bs[nn][kq] = rb[q];
        }
    };
    if (kb < ke) fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += GT_K) {
        stage();
        __syncthreads();
        if (k0 + GT_K < ke) fetch(k0 + GT_K);
#pragma unroll
        for (int ks = 0; ks < GT_K; ks += 8) {
            uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gid;
                const float v[4] = {As[r][ks + tig], As[r + 8][ks + tig], As[r][ks + tig + 4], As[r + 8][ks + tig + 4]};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (A_EXACT) {
                        ah[i][q] = __float_as_uint(v[q]);
                        al[i][q] = 0u;
                    } else {
                        split_tf32(v[q], ah[i][q], al[i][q]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + gid;
                const float v[2] = {Bs[c][ks + tig], Bs[c][ks + tig + 4]};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    if (B_EXACT) {
                        bh[j][q] = __float_as_uint(v[q]);
                        bl[j][q] = 0u;
                    } else {
                        split_tf32(v[q], bh[j][q], bl[j][q]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // small terms first, then the leading product
                    if (!A_EXACT) mma_tf32(acc[i][j], al[i], bh[j]);
                    if (!B_EXACT) mma_tf32(acc[i][j], ah[i], bl[j]);
                    mma_tf32(acc[i][j], ah[i], bh[j]);
                }
        }
        __syncthreads();
    }
    // accumulator fragment: e = 0, 1 at row gid, columns 2 tig, 2 tig + 1; e = 2, 3 at row gid + 8
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + i * 16 + gid + (e >> 1) * 8;
                const int n = n0 + wn + j * 8 + tig * 2 + (e & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][e];
                if (EPI == EPI_BIAS || EPI == EPI_BIAS_RELU) v += __bfloat162float(bias[n]);
                if (EPI == EPI_BIAS_RELU) v = fmaxf(v, 0.f);
                if (EPI == EPI_MASK) v = mask[(size_t)m * ldm + n] > 0.f ? v : 0.f;
                Cz[(size_t)m * ldc + n] = v;
            }
}

// C = sum of the split-K partials in split order (a fixed order: results do not depend on timing).
__global__ void k_sum_splits(const float* part, int splits, long long n, float* C) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = part[i];
        for (int z = 1; z < splits; ++z) s += part[(size_t)z * n + i];
        C[i] = s;
    }
}

// One CTA per 64 x 64 output tile over all of K.
template <typename TAE, typename TBE, bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const TAE* A, int lda, const TBE* B, int ldb, float* C, int ldc,
                 const __nv_bfloat16* bias, const float* mask, int ldm, cudaStream_t s) {
    dim3 grid((N + GT_N - 1) / GT_N, (M + GT_M - 1) / GT_M, 1);
    k_gemm<TAE, TBE, TA, TB, EPI><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mask, ldm,
                                                        (K + GT_K - 1) / GT_K * GT_K);
    return cudaGetLastError();
}

// Split-K for a product with few output tiles and a long K (the weight gradients, K = rows): up to
// `splits` CTAs per tile, each over a 16-aligned share of K, their partials summed by k_sum_splits.
// work: splits * M * N floats; C is a dense M x N array.
template <typename TAE, typename TBE, bool TA, bool TB>
cudaError_t gemm_splitk(int M, int N, int K, const TAE* A, int lda, const TBE* B, int ldb, float* C, float* work,
                        int splits, cudaStream_t s) {
    const int chunk = ((K + splits - 1) / splits + GT_K - 1) / GT_K * GT_K;
    splits = chunk > 0 ? (K + chunk - 1) / chunk : 1;
    if (splits <= 1) return gemm<TAE, TBE, TA, TB, EPI_STORE>(M, N, K, A, lda, B, ldb, C, N, nullptr, nullptr, 0, s);
    dim3 grid((N + GT_N - 1) / GT_N, (M + GT_M - 1) / GT_M, splits);
    k_gemm<TAE, TBE, TA, TB, EPI_STORE><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, work, N, nullptr, nullptr, 0, chunk);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)M * N;
    k_sum_splits<<<(unsigned)std::min<long long>((n + 255) / 256, 1024), 256, 0, s>>>(work, splits, n, C);
    return cudaGetLastError();
}

// dY = 2 (x[:, :8] + y - target) / n and per-block partial sums of the squared error.
__global__ void k_mse(const float* X, int n_in, const float* Y, const float* T, float* dY, int n, int n_out,
                      double* part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)n * n_out;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n_out, c = i % n_out;
        const float d = X[r * n_in + c] + Y[i] - T[i];
        dY[i] = 2.f * d / (float)n;
        s += (double)d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_sum_parts(const double* part, int np, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < np; ++i) s += part[i];
        *out = s / n;
    }
}

// db[c] = sum_r g[r][c]: 32 columns per block, 8 row groups, fixed-order combination.
__global__ void k_colsum(const float* g, int n, int cols, float* db) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + (threadIdx.x & 31), grp = threadIdx.x >> 5;
    float s = 0.f;
    if (c < cols)
        for (int r = grp; r < n; r += 8) s += g[(size_t)r * cols + c];
    red[grp][threadIdx.x & 31] = s;
    __syncthreads();
    if (grp == 0 && c < cols) {
        float t = 0.f;
        for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
        db[c] = t;
    }
}

// AdamW (decoupled decay) on the float32 master weights; refresh the bfloat16 copies.
__global__ void k_adamw(float* w, __nv_bfloat16* wb, float* m, float* v, const float* g, long long np, float lr,
                        float b1, float b2, float c1, float c2, float eps, float wd) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float upd = (mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i];
        const float wi = w[i] - lr * upd;
        w[i] = wi;
        wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* wb, long long np) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void k_add_rows(const float* X, int n_in, const float* Y, float* out, long long n) {
    // out[r][c] = X[r][c] + Y[r][c] for the 8 Jones entries of a row
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * 8; i += (long long)gridDim.x * blockDim.x)
        out[i] = X[(i / 8) * n_in + (i % 8)] + Y[i];
}

// Warm-start features: rows (a, k, p) of [J_prev, B_f Z_prev, x_f].
__global__ void k_ws_features(const float* J, const float* BZ, const double* xf, int K, int N, long long rows,
                              float* X) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(r / ((long long)K * N));
        float* x = X + r * 17;
        for (int i = 0; i < 8; ++i) {
            x[i] = J[r * 8 + i];
            x[8 + i] = BZ[r * 8 + i];
        }
        x[16] = (float)xf[a];
    }
}

// Per agent keep the network's start only where it lowers L_i (the previous solution is the fallback).
__global__ void k_ws_select(const float* J_mlp, const float* J_prev, const double* L_mlp, const double* L_prev,
                            int KN8, int A, float* J_out, int* chose) {
    const int a = blockIdx.x;
    if (a >= A) return;
    const bool use = isfinite(L_mlp[a]) && L_mlp[a] < L_prev[a];
    if (threadIdx.x == 0 && chose) chose[a] = use ? 1 : 0;
    const float* src = (use ? J_mlp : J_prev) + (size_t)a * KN8;
    for (int i = threadIdx.x; i < KN8; i += blockDim.x) J_out[(size_t)a * KN8 + i] = src[i];
}

unsigned grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)std::max(1LL, std::min(b, 4096LL));
}

}  // namespace

struct MlpNet {
    int n_in = 17, width = 256, depth = 3, n_out = 8;
    std::vector<int> in_dim, out_dim;
    std::vector<long long> off_w, off_b;
    long long n_params = 0;
    float* master = nullptr;
    __nv_bfloat16* wb = nullptr;
    float *m = nullptr, *v = nullptr, *grad = nullptr;
    long long t = 0;
    int cap = 0;
    std::vector<float*> act;
    float *X = nullptr, *T = nullptr, *g1 = nullptr, *g2 = nullptr, *pred = nullptr;
    float* splitk = nullptr;  // split-K partials of the weight gradients: SPLITK_MAX x the largest layer
    int sms = 1;              // SM count of the device
    double *part = nullptr, *loss = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
};

namespace {

cudaError_t ensure_cap(MlpNet* n, int rows) {
    if (rows <= n->cap) return cudaSuccess;
    cudaStreamSynchronize(n->stream);
    for (float* p : n->act) cudaFree(p);
    n->act.clear();
    cudaFree(n->X); cudaFree(n->T); cudaFree(n->g1); cudaFree(n->g2); cudaFree(n->pred);
    const int wmax = std::max(n->width, std::max(n->n_in, n->n_out));
    cudaError_t e = cudaSuccess;
    for (size_t l = 0; l < n->out_dim.size() && e == cudaSuccess; ++l) {
        float* p = nullptr;
        e = cudaMalloc(&p, (size_t)rows * n->out_dim[l] * sizeof(float));
        n->act.push_back(p);
    }
    if (e == cudaSuccess) e = cudaMalloc(&n->X, (size_t)rows * n->n_in * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->T, (size_t)rows * n->n_out * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->g1, (size_t)rows * wmax * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->g2, (size_t)rows * wmax * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->pred, (size_t)rows * 8 * sizeof(float));
    if (e == cudaSuccess) n->cap = rows;
    return e;
}

cudaError_t forward(MlpNet* n, const float* X, int rows) {
    const float* h = X;
    const int L = (int)n->out_dim.size();
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        const __nv_bfloat16* W = n->wb + n->off_w[l];
        const __nv_bfloat16* b = n->wb + n->off_b[l];
        if (l < L - 1)
            e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS_RELU>(rows, n->out_dim[l], n->in_dim[l], h, n->in_dim[l], W,
                                                                       n->in_dim[l], n->act[l], n->out_dim[l], b, nullptr, 0,
                                                                       n->stream);
        else
            e = gemm<float, __nv_bfloat16, false, true, EPI_BIAS>(rows, n->out_dim[l], n->in_dim[l], h, n->in_dim[l], W,
                                                                  n->in_dim[l], n->act[l], n->out_dim[l], b, nullptr, 0,
                                                                  n->stream);
        h = n->act[l];
    }
    return e;
}

// Gradient of the mean squared error of x[:, :8] + y against T into n->grad; loss into n->loss.
cudaError_t backward(MlpNet* n, const float* X, const float* T, int rows) {
    const int L = (int)n->out_dim.size();
    const unsigned nb = grid_for((long long)rows * n->n_out);
    k_mse<<<nb, 256, 0, n->stream>>>(X, n->n_in, n->act[L - 1], T, n->g1, rows, n->n_out, n->part);
    k_sum_parts<<<1, 32, 0, n->stream>>>(n->part, (int)nb, rows, n->loss);
    cudaError_t e = cudaGetLastError();
    float* g = n->g1;
    float* other = n->g2;
    for (int l = L - 1; l >= 0 && e == cudaSuccess; --l) {
        const float* h_in = l == 0 ? X : n->act[l - 1];
        const int in = n->in_dim[l], out = n->out_dim[l];
        // dW = g^T h_in  (out x in): few output tiles over a long K (the rows), so split K
        const int tiles = ((out + GT_M - 1) / GT_M) * ((in + GT_N - 1) / GT_N);
        const int splits = std::max(1, std::min(SPLITK_MAX, 2 * n->sms / tiles));  // about two CTAs per SM
        e = gemm_splitk<float, float, true, false>(out, in, rows, g, out, h_in, in, n->grad + n->off_w[l], n->splitk,
                                                   splits, n->stream);
        if (e != cudaSuccess) break;
        k_colsum<<<(out + 31) / 32, 256, 0, n->stream>>>(g, rows, out, n->grad + n->off_b[l]);
        e = cudaGetLastError();
        if (l > 0 && e == cudaSuccess) {
            // g_prev = (g W) masked by the ReLU of the layer below
            e = gemm<float, __nv_bfloat16, false, false, EPI_MASK>(rows, in, out, g, out, n->wb + n->off_w[l], in, other, in,
                                                                   nullptr, n->act[l - 1], in, n->stream);
            std::swap(g, other);
        }
    }
    return e;
}

}  // namespace
}  // namespace calib

using calib::MlpNet;

struct calib_mlp {
    MlpNet net;
};

namespace {
int mfail(int code, const std::string& m) {
    calib::set_last_error(m);
    return code;
}
#define MCK(expr)                                                                                  \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return mfail(CALIB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)
}  // namespace

extern "C" {

int calib_mlp_create(calib_mlp** out, int n_in, int width, int depth, int n_out, void* cuda_stream) {
    if (!out) return mfail(CALIB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in != 17 || n_out != 8) return mfail(CALIB_EINVAL, "the warm-start rows have 17 inputs and 8 outputs");
    if (width < 1 || width > 4096 || depth < 1 || depth > 16) return mfail(CALIB_EINVAL, "width in [1,4096], depth in [1,16]");
    calib_mlp* h = new calib_mlp();
    MlpNet* n = &h->net;
    n->n_in = n_in;
    n->width = width;
    n->depth = depth;
    n->n_out = n_out;
    for (int l = 0; l <= depth; ++l) {
        n->in_dim.push_back(l == 0 ? n_in : width);
        n->out_dim.push_back(l == depth ? n_out : width);
    }
    long long off = 0;
    for (size_t l = 0; l < n->in_dim.size(); ++l) {
        n->off_w.push_back(off);
        off += (long long)n->in_dim[l] * n->out_dim[l];
        n->off_b.push_back(off);
        off += n->out_dim[l];
    }
    n->n_params = off;
    cudaError_t e = cudaSuccess;
    if (cuda_stream) {
        n->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
        n->own_stream = true;
    }
    if (e == cudaSuccess) e = cudaMalloc(&n->master, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->wb, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&n->m, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->v, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->grad, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&n->part, 4096 * sizeof(double));
    long long largest = 0;
    for (size_t l = 0; l < n->in_dim.size(); ++l) largest = std::max(largest, (long long)n->in_dim[l] * n->out_dim[l]);
    if (e == cudaSuccess) e = cudaMalloc(&n->splitk, (size_t)calib::SPLITK_MAX * largest * sizeof(float));
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&n->loss, sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(n->master, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->wb, 0, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(n->m, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(n->v, 0, off * sizeof(float));
    if (e != cudaSuccess) {
        calib_mlp_destroy(h);
        return mfail(CALIB_ENOMEM, std::string("calib_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = h;
    return CALIB_OK;
}

long long calib_mlp_num_params(calib_mlp* h) { return h ? h->net.n_params : 0; }

int calib_mlp_set_weights(calib_mlp* h, const float* w, int ptr_kind) {
    if (!h || !w) return mfail(CALIB_EINVAL, "mlp and w are required");
    MlpNet* n = &h->net;
    MCK(cudaMemcpyAsync(n->master, w, n->n_params * sizeof(float),
                        ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->stream));
    calib::k_to_bf16<<<calib::grid_for(n->n_params), 256, 0, n->stream>>>(n->master, n->wb, n->n_params);
    MCK(cudaGetLastError());
    MCK(cudaMemsetAsync(n->m, 0, n->n_params * sizeof(float), n->stream));
    MCK(cudaMemsetAsync(n->v, 0, n->n_params * sizeof(float), n->stream));
    n->t = 0;
    if (ptr_kind == 0) MCK(cudaStreamSynchronize(n->stream));
    return CALIB_OK;
}

int calib_mlp_get_weights(calib_mlp* h, float* w, int ptr_kind) {
    if (!h || !w) return mfail(CALIB_EINVAL, "mlp and w are required");
    MlpNet* n = &h->net;
    MCK(cudaMemcpyAsync(w, n->master, n->n_params * sizeof(float),
                        ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
    if (ptr_kind == 0) MCK(cudaStreamSynchronize(n->stream));
    return CALIB_OK;
}

int calib_mlp_forward(calib_mlp* h, const float* X, float* Y, int rows, int ptr_kind) {
    if (!h || !X || !Y || rows < 1) return mfail(CALIB_EINVAL, "mlp, X, Y and rows >= 1 are required");
    MlpNet* n = &h->net;
    MCK(calib::ensure_cap(n, rows));
    const float* Xd = X;
    if (ptr_kind == 0) {
        MCK(cudaMemcpyAsync(n->X, X, (size_t)rows * n->n_in * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        Xd = n->X;
    }
    MCK(calib::forward(n, Xd, rows));
    MCK(cudaMemcpyAsync(Y, n->act.back(), (size_t)rows * n->n_out * sizeof(float),
                        ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->stream));
    if (ptr_kind == 0) MCK(cudaStreamSynchronize(n->stream));
    return CALIB_OK;
}

int calib_mlp_grad(calib_mlp* h, const float* X, const float* T, int rows, float* grad, double* loss, int ptr_kind) {
    if (!h || !X || !T || rows < 1) return mfail(CALIB_EINVAL, "mlp, X, T and rows >= 1 are required");
    MlpNet* n = &h->net;
    MCK(calib::ensure_cap(n, rows));
    const float *Xd = X, *Td = T;
    if (ptr_kind == 0) {
        MCK(cudaMemcpyAsync(n->X, X, (size_t)rows * n->n_in * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        MCK(cudaMemcpyAsync(n->T, T, (size_t)rows * n->n_out * sizeof(float), cudaMemcpyHostToDevice, n->stream));
        Xd = n->X;
        Td = n->T;
    }
    MCK(calib::forward(n, Xd, rows));
    MCK(calib::backward(n, Xd, Td, rows));
    const cudaMemcpyKind k = ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (grad) MCK(cudaMemcpyAsync(grad, n->grad, n->n_params * sizeof(float), k, n->stream));
    if (loss) MCK(cudaMemcpyAsync(loss, n->loss, sizeof(double), k, n->stream));
    if (ptr_kind == 0) MCK(cudaStreamSynchronize(n->stream));
    return CALIB_OK;
}

int calib_mlp_train_step(calib_mlp* h, const float* X, const float* T, int rows, float lr, float weight_decay,
                         double* loss, int ptr_kind) {
    if (!h) return mfail(CALIB_EINVAL, "mlp is NULL");
    MlpNet* n = &h->net;
    int rc = calib_mlp_grad(h, X, T, rows, nullptr, nullptr, ptr_kind);
    if (rc) return rc;
    n->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - (float)std::pow((double)b1, (double)n->t), c2 = 1.f - (float)std::pow((double)b2, (double)n->t);
    calib::k_adamw<<<calib::grid_for(n->n_params), 256, 0, n->stream>>>(n->master, n->wb, n->m, n->v, n->grad, n->n_params,
                                                                         lr, b1, b2, c1, c2, 1e-8f, weight_decay);
    MCK(cudaGetLastError());
    if (loss) {
        MCK(cudaMemcpyAsync(loss, n->loss, sizeof(double), ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            n->stream));
        if (ptr_kind == 0) MCK(cudaStreamSynchronize(n->stream));
    }
    return CALIB_OK;
}

void calib_mlp_destroy(calib_mlp* h) {
    if (!h) return;
    MlpNet* n = &h->net;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (float* p : n->act) cudaFree(p);
    for (void* p : {(void*)n->master, (void*)n->wb, (void*)n->m, (void*)n->v, (void*)n->grad, (void*)n->splitk, (void*)n->X, (void*)n->T,
                    (void*)n->g1, (void*)n->g2, (void*)n->pred, (void*)n->part, (void*)n->loss})
        if (p) cudaFree(p);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
    delete h;
}

}  // extern "C"

// ---- warm start of a calibration context (needs the context internals: capi.cu helpers)
namespace calib {
cudaError_t mlp_warm_rows(calib_mlp* h, const float* J_prev, const float* BZ, const double* xf, int K, int N, int A,
                          float* J_mlp, cudaStream_t s) {
    MlpNet* n = &h->net;
    const long long rows = (long long)A * K * N;
    cudaError_t e = ensure_cap(n, (int)rows);
    if (e != cudaSuccess) return e;
    k_ws_features<<<grid_for(rows), 256, 0, s>>>(J_prev, BZ, xf, K, N, rows, n->X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cudaStream_t keep = n->stream;
    n->stream = s;
    e = forward(n, n->X, (int)rows);
    n->stream = keep;
    if (e != cudaSuccess) return e;
    k_add_rows<<<grid_for(rows * 8), 256, 0, s>>>(n->X, n->n_in, n->act.back(), J_mlp, rows);
    return cudaGetLastError();
}
cudaError_t launch_ws_features(const float* J, const float* BZ, const double* xf, int K, int N, long long rows, float* X,
                               cudaStream_t s) {
    k_ws_features<<<grid_for(rows), 256, 0, s>>>(J, BZ, xf, K, N, rows, X);
    return cudaGetLastError();
}
cudaError_t mlp_warm_select(const float* J_mlp, const float* J_prev, const double* L_mlp, const double* L_prev, int KN8,
                            int A, float* J_out, int* chose, cudaStream_t s) {
    k_ws_select<<<A, 256, 0, s>>>(J_mlp, J_prev, L_mlp, L_prev, KN8, A, J_out, chose);
    return cudaGetLastError();
}
}  // namespace calib
