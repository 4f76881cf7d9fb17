// Hessian pass of the J-update on the per-baseline sufficient statistics (Section 3, Eq. HessL):
// the one-thread-per-slot kernel used for K <= 5 (the layout, partition and copy ring are those of
// the sweeps in ss.cu; see there for the identities).
#include "ss_common.cuh"

namespace calib {
namespace {

using namespace ss;

// Hessian pass with one thread per slot (both rows of the 2x2 blocks), for K <= HV1_KMAX: the second
// station's rows of J and eta are read from shared memory once per slot instead of once per row
// thread, the first station's other row is in registers, and no partner exchange is needed; the
// price is twice the registers per thread (both rows of J, eta and the first-station sums).
// Same partition, copy ring, statistics layout and partial layout as k_ss_sweep.
// Stage layout: [S: n2][KK] float2.
// 64 threads (N <= 64) at up to 255 registers: 4 CTAs, 8 warps per SM.
template <int KB>
__global__ void __launch_bounds__(128, 2) k_ss_hessvec(const SSArgs a, const int stage_bytes) {
    constexpr int NST = nst<true>();
    extern __shared__ __align__(128) unsigned char smem[];
    const int N = a.N, D = a.D, NP = a.NP;
    constexpr int K = KB;
    const int KK = K * (K + 1) / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid;
    const int KN2 = K * N * 2;
    const bool own = g < N;

    unsigned char* stage = smem;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NST * stage_bytes);
    // [K][2 rows][N]: consecutive threads read consecutive 16-byte entries (no bank conflicts)
    float4* Js = reinterpret_cast<float4*>(smem + NST * stage_bytes + BAR_BYTES);
    float4* Es = Js + KN2;
    float4* accs = Es + KN2;

    const long long W = (long long)a.A * D, G = gridDim.x;
    const long long i0 = (long long)blockIdx.x * W / G;
    const int S = (int)((long long)(blockIdx.x + 1) * W / G - i0);
    const int ag0 = (int)(i0 / D), d0 = (int)(i0 - (long long)ag0 * D);

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    int iss_ag = ag0, iss_d = d0;
    const uint64_t pol = tid == 0 ? l2_evict_first() : 0ull;
    auto issue = [&](int s2) {
        const size_t blk = ((size_t)iss_ag * D + iss_d) * NP;
        const int n = (2 * (iss_d + 1) == N) ? N / 2 : N;
        const int n2 = (n + 1) & ~1;
        if (++iss_d == D) { iss_d = 0; ++iss_ag; }
        const uint32_t sb = (uint32_t)(n2 * KK * 8);
        uint64_t* b = &bar[s2 % NST];
        mbar_expect_tx(b, sb);
        bulk_g2s_stream(stage + (s2 % NST) * stage_bytes, a.S + blk * KK, sb, b, pol);
    };
    if (tid == 0)
        for (int s2 = 0; s2 < min(NST - 1, S); ++s2) issue(s2);
    // Everything above reads only the statistics; J, eta (or J') and the partial buffers belong to
    // the preceding kernels of the chain (programmatic dependent launch).
    griddep_wait();
    griddep_launch_dependents();

    float4 Jf[KB][2], Ef[KB][2], A1[KB][2];  // station g's rows of J and eta; its first-station sums
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int r = 0; r < 2; ++r) Jf[k][r] = Ef[k][r] = A1[k][r] = z4;

    auto flush = [&](int ag) {
        const long long piece = blockIdx.x - cta_of_item((long long)ag * D, W, G);
        const size_t slot_p = (size_t)ag * a.part_stride + (size_t)piece;
        float4* out = reinterpret_cast<float4*>(a.part) + slot_p * KN2;
        if (own) {
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 w = accs[(k * 2 + r) * N + g];
                    out[(k * N + g) * 2 + r] = make_float4(A1[k][r].x + w.x, A1[k][r].y + w.y, A1[k][r].z + w.z, A1[k][r].w + w.w);
                }
            }
        }
    };

    int agent = -1, ag = ag0, dg = d0;
    bool fresh = false;
    for (int s = 0; s < S; ++s) {
        if (ag != agent) {
            if (agent >= 0) {
                __syncthreads();
                flush(agent);
                __syncthreads();
            }
            agent = ag;
            fresh = true;
            const float4* Jg = reinterpret_cast<const float4*>(a.J) + (size_t)ag * KN2;
            const float4* Eg = reinterpret_cast<const float4*>(a.eta) + (size_t)ag * KN2;
            for (int i = tid; i < KN2; i += nthr) {  // global [K][N][2] -> shared [K][2][N]
                const int r = i & 1, kn = i >> 1, kk = kn / N, st = kn - kk * N;
                const int o = (kk * 2 + r) * N + st;
                Js[o] = __ldg(Jg + i);
                Es[o] = __ldg(Eg + i);
                accs[i] = z4;
            }
        }
        const int d = dg + 1;
        if (++dg == D) { dg = 0; ++ag; }
        const bool ok = mbar_wait_bounded(&bar[s % NST], (uint32_t)((s / NST) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.status, STATUS_TIMEOUT);
                const int last = min(S - 1, s + NST - 1);
                for (int s2 = s; s2 <= last; ++s2) mbar_wait_bounded(&bar[s2 % NST], (uint32_t)((s2 / NST) & 1));
            }
            return;
        }
        if (tid == 0 && s + NST - 1 < S) {
            fence_proxy_async_smem();
            issue(s + NST - 1);
        }
        if (fresh) {
            fresh = false;
            if (own) {
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k >= K) continue;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        Jf[k][r] = Js[(k * 2 + r) * N + g];
                        Ef[k][r] = Es[(k * 2 + r) * N + g];
                        A1[k][r] = z4;
                    }
                }
            }
        }
        const int n = (2 * d == N) ? N / 2 : N;
        if (g >= n) continue;
        const float2* Ss = reinterpret_cast<const float2*>(stage + (s % NST) * stage_bytes) + (size_t)g * KK;
        const int second = (g + d < N) ? g + d : g + d - N;
        // X_k = (S Q)_k, entries [row][column] at 2 row + column
        float2 X[KB][4];
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) X[k][e] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KB; ++l) {
            if (l >= K) continue;
            // Q_l = eta_f J_s^H + J_f eta_s^H; (A B^H)[r][c] = A[r][0] conj(B[c][0]) + A[r][1] conj(B[c][1])
            const float4 js0 = Js[2 * l * N + second], js1 = Js[(2 * l + 1) * N + second];
            const float4 es0 = Es[2 * l * N + second], es1 = Es[(2 * l + 1) * N + second];
            const float2 z2 = make_float2(0.f, 0.f);
            float2 q[4];
            q[0] = cdot2_acc(cdot2_acc(z2, Ef[l][0], js0), Jf[l][0], es0);
            q[1] = cdot2_acc(cdot2_acc(z2, Ef[l][0], js1), Jf[l][0], es1);
            q[2] = cdot2_acc(cdot2_acc(z2, Ef[l][1], js0), Jf[l][1], es0);
            q[3] = cdot2_acc(cdot2_acc(z2, Ef[l][1], js1), Jf[l][1], es1);
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
                const int lo = k < l ? k : l, hi = k < l ? l : k;
                float2 skl = Ss[lo * K - lo * (lo - 1) / 2 + (hi - lo)];
                if (k > l) skl.y = -skl.y;
#pragma unroll
                for (int e = 0; e < 4; ++e) cmac(X[k][e], skl, q[e]);
            }
        }
        // Station terms. First station (registers): (X_k J_s)[r][.] = X[r][0] J_s[0][.] + X[r][1] J_s[1][.].
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k >= K) continue;
            const float4 s0 = Js[2 * k * N + second], s1 = Js[(2 * k + 1) * N + second];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 a0 = cmul2_acc(make_float2(A1[k][r].x, A1[k][r].y), 1.f, X[k][2 * r], make_float2(s0.x, s0.y),
                                            X[k][2 * r + 1], make_float2(s1.x, s1.y));
                const float2 a1 = cmul2_acc(make_float2(A1[k][r].z, A1[k][r].w), 1.f, X[k][2 * r], make_float2(s0.z, s0.w),
                                            X[k][2 * r + 1], make_float2(s1.z, s1.w));
                A1[k][r] = make_float4(a0.x, a0.y, a1.x, a1.y);
            }
        }
        // Second station (shared): (X_k^H J_f)[r][.] = conj(X[0][r]) J_f[0][.] + conj(X[1][r]) J_f[1][.].
        // Every sum is read before any is written: the compiler cannot tell the directions'
        // addresses apart and would otherwise wait for each store before the next load.
        float4 t2[KB][2];
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int r = 0; r < 2; ++r) t2[k][r] = k < K ? accs[(k * 2 + r) * N + second] : z4;
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k >= K) continue;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float2 b0 = cmul2c_acc(make_float2(t2[k][r].x, t2[k][r].y), 1.f, X[k][r], make_float2(Jf[k][0].x, Jf[k][0].y),
                                             X[k][2 + r], make_float2(Jf[k][1].x, Jf[k][1].y));
                const float2 b1 = cmul2c_acc(make_float2(t2[k][r].z, t2[k][r].w), 1.f, X[k][r], make_float2(Jf[k][0].z, Jf[k][0].w),
                                             X[k][2 + r], make_float2(Jf[k][1].z, Jf[k][1].w));
                accs[(k * 2 + r) * N + second] = make_float4(b0.x, b0.y, b1.x, b1.y);
            }
        }
    }
    if (agent >= 0) {
        __syncthreads();
        flush(agent);
    }
}


template <int KB>
cudaError_t prep_hv1() {
    return cudaFuncSetAttribute(k_ss_hessvec<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}


template <int KB>
cudaError_t go_hv1(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s) {
    return launch_k(a.pdl != 0, k_ss_hessvec<KB>, grid, threads, smem, s, a, sb);
}

cudaError_t dispatch_hv1(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s) {
    static_assert(HV1_KMAX == 5, "dispatch_hv1 covers K = 1 .. 5");
    switch (a.K) {
        case 1: return go_hv1<1>(a, grid, threads, smem, sb, s);
        case 2: return go_hv1<2>(a, grid, threads, smem, sb, s);
        case 3: return go_hv1<3>(a, grid, threads, smem, sb, s);
        case 4: return go_hv1<4>(a, grid, threads, smem, sb, s);
        default: return go_hv1<5>(a, grid, threads, smem, sb, s);
    }
}

}  // namespace

cudaError_t prepare_ss_hessvec_kernels() {
    cudaError_t e = prep_hv1<1>();
    if (e == cudaSuccess) e = prep_hv1<2>();
    if (e == cudaSuccess) e = prep_hv1<3>();
    if (e == cudaSuccess) e = prep_hv1<4>();
    if (e == cudaSuccess) e = prep_hv1<5>();
    return e;
}

cudaError_t launch_ss_hessvec1(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s) {
    return dispatch_hv1(a, grid, threads, smem, sb, s);
}

}  // namespace calib
