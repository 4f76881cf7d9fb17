// SAGE decomposition of the K-direction J-update (step D1 of Section 3): the directions are
// solved one at a time; for direction k the expectation step removes the other directions' models
// from the data, V_k = V - sum_{l != k} J_pl C_pql J_ql^H, and the maximisation step minimises
// direction k's own Lagrangian ||V_k - J_pk C_pqk J_qk^H||^2 + Re tr(Y_k^H (J_k - BZ_k)) +
// rho_k/2 ||J_k - BZ_k||^2 over J_k (by RTR, the paper's solver).
//
// On the per-baseline sufficient statistics the expectation step is exact and needs no pass over
// the visibilities: sum_t conj(c_tk) V_k(t) = U_k - sum_{l != k} S_kl P_l with P_l = J_pl J_ql^H,
// and sum_t |c_tk|^2 = S_kk. So direction k's problem is a one-direction problem with statistics
// U' = U_k - sum_{l != k} S_kl P_l and S' = S_kk in the same full circulant layout, solved by the
// same sweeps and per-agent kernels with K = 1 on gathered copies of J_k, Y_k and B Z_k.
#include "calib_internal.cuh"

namespace calib {
namespace {

constexpr int SG_THREADS = 256;

// One thread per slot position of the full circulant layout: U' and S' of direction k.
__global__ void __launch_bounds__(SG_THREADS) k_sage_stats(const float2* __restrict__ U, const float2* __restrict__ S,
                                                          const float* __restrict__ J, float2* __restrict__ U1,
                                                          float2* __restrict__ S1, int A, int D, int NP, int K, int N,
                                                          int k) {
    const long long pos = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= (long long)A * D * NP) return;
    const int i = (int)(pos % NP);
    const long long ad = pos / NP;
    const int d = (int)(ad % D) + 1, a = (int)(ad / D);
    const int n = (2 * d == N) ? N / 2 : N;  // slots of this diagonal
    const int KK = K * (K + 1) / 2;
    float2 u[4];
    float2 skk = make_float2(0.f, 0.f);
    if (i < n) {
        const float2* up = U + pos * K * 4 + (size_t)k * 4;
        const float2* sp = S + pos * KK;
#pragma unroll
        for (int e = 0; e < 4; ++e) u[e] = up[e];
        skk = sp[k * K - k * (k - 1) / 2];
        const int f = i, s = (i + d < N) ? i + d : i + d - N;  // first and second station
        for (int l = 0; l < K; ++l) {
            if (l == k) continue;
            const int lo = k < l ? k : l, hi = k < l ? l : k;
            float2 skl = sp[lo * K - lo * (lo - 1) / 2 + (hi - lo)];
            if (k > l) skl.y = -skl.y;  // S_kl = conj(S_lk) below the diagonal
            const float2* jf = reinterpret_cast<const float2*>(J) + ((size_t)a * K + l) * N * 4 + (size_t)f * 4;
            const float2* js = reinterpret_cast<const float2*>(J) + ((size_t)a * K + l) * N * 4 + (size_t)s * 4;
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    // P[r][c] = sum_m J_f[r][m] conj(J_s[c][m])
                    float pr = 0.f, pi = 0.f;
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const float2 x = jf[r * 2 + m], y = js[c * 2 + m];
                        pr = fmaf(x.x, y.x, fmaf(x.y, y.y, pr));
                        pi = fmaf(x.y, y.x, fmaf(-x.x, y.y, pi));
                    }
                    // u -= S_kl P
                    float2& o = u[r * 2 + c];
                    o.x -= skl.x * pr - skl.y * pi;
                    o.y -= skl.x * pi + skl.y * pr;
                }
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) u[e] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) U1[pos * 4 + e] = u[e];
    S1[pos] = skk;
}

// Copies of direction k's J (also as the trial point J' = J), Y and B Z: [A][N][8] from [A][K][N][8].
__global__ void __launch_bounds__(SG_THREADS) k_sage_gather(const float* __restrict__ J, const float* __restrict__ Y,
                                                           const float* __restrict__ BZ, float* __restrict__ J1,
                                                           float* __restrict__ Jt1, float* __restrict__ Y1,
                                                           float* __restrict__ BZ1, int A, int K, int N, int k) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n8 = (long long)N * 8;
    if (i >= (long long)A * n8) return;
    const long long a = i / n8, r = i - a * n8;
    const size_t src = ((size_t)a * K + k) * n8 + r;
    const float j = J[src];
    J1[i] = j;
    Jt1[i] = j;
    Y1[i] = Y[src];
    BZ1[i] = BZ[src];
}

__global__ void __launch_bounds__(SG_THREADS) k_sage_scatter(const float* __restrict__ J1, float* __restrict__ J, int A,
                                                            int K, int N, int k) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n8 = (long long)N * 8;
    if (i >= (long long)A * n8) return;
    const long long a = i / n8, r = i - a * n8;
    J[((size_t)a * K + k) * n8 + r] = J1[i];
}

unsigned blocks_for(long long n) { return (unsigned)((n + SG_THREADS - 1) / SG_THREADS); }

}  // namespace

cudaError_t launch_sage_prepare(const SageArgs& g, int k, cudaStream_t s) {
    const long long npos = (long long)g.A * g.D * g.NP;
    k_sage_stats<<<blocks_for(npos), SG_THREADS, 0, s>>>(g.U, g.S, g.J, g.U1, g.S1, g.A, g.D, g.NP, g.K, g.N, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sage_gather<<<blocks_for((long long)g.A * g.N * 8), SG_THREADS, 0, s>>>(g.J, g.Y, g.BZ, g.J1, g.Jt1, g.Y1, g.BZ1,
                                                                            g.A, g.K, g.N, k);
    return cudaGetLastError();
}

cudaError_t launch_sage_scatter(const SageArgs& g, int k, cudaStream_t s) {
    k_sage_scatter<<<blocks_for((long long)g.A * g.N * 8), SG_THREADS, 0, s>>>(g.J1, g.J_out, g.A, g.K, g.N, k);
    return cudaGetLastError();
}

}  // namespace calib
