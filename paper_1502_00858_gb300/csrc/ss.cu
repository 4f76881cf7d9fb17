// Baseline sweeps of the J-update on per-baseline sufficient statistics (Section 3, Eq. M1).
//
// Because C = c I_2 (Eq. coh) and J is constant over a solution interval (Section 2), every sum over
// the samples of a baseline factors through U_k = sum_t conj(c_tk) V_t and S_kl = sum_t conj(c_tk) c_tl:
//   Hessian pass:  sum_t conj(c_tk) dM_t = sum_l S_kl Q_l,  Q_l = eta_pl J_ql^H + J_pl eta_ql^H,
//                  so the station terms of H_GN eta (Eq. HessL) are U'_k J_qk and U'_k^H J_pk, U'_k = S Q;
//   trial pass:    W_k = sum_t conj(c_tk) R_t = U_k - sum_l S_kl P_l (P_l = J_pl J_ql^H) at J, and at
//                  J' = J + x: W'_k = W_k - sum_l S_kl dP_l with the exact model change
//                  dP_l = x_pl J_ql^H + J_pl x_ql^H + x_pl x_ql^H; the data-cost decrease is
//                  g(J) - g(J') = sum_k Re <dP_k, 2 W_k - (S dP)_k> (Frobenius inner product).
// The identities are exact; the per-pass work and traffic no longer depend on the number of samples.
// Mapping, per-station scatter and the bounded mbarrier/TMA-bulk ring follow sweep.cu: one CTA per
// (agent, chunk of circulant diagonals), one stage per diagonal, four threads per slot (one per
// correlation), two barrier-separated shared-memory phases per diagonal (no atomics).
#include "calib_internal.cuh"

namespace calib {
namespace {

constexpr int NST = 2;   // one stage = one whole diagonal; one stage of prefetch hides the bulk-copy latency
constexpr int BAR_BYTES = 64;  // barrier area, keeps the rows below 16-byte aligned

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_BUDGET_CYCLES) return false;
    }
    return true;
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float2 cmul_cb(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
__device__ __forceinline__ float2 cmul_ca(float2 a, float2 b) { return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }
// acc += s * q
__device__ __forceinline__ void cmac(float2& acc, float2 s, float2 q) {
    acc.x = fmaf(s.x, q.x, fmaf(-s.y, q.y, acc.x));
    acc.y = fmaf(s.x, q.y, fmaf(s.y, q.x, acc.y));
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// KB: register bucket; EXACT: K == KB, so every loop bound and packed-S index is a constant.
template <int KB, bool HV, bool EXACT>
__global__ void __launch_bounds__(512) k_ss_sweep(const SSArgs a, const int stage_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int agent = blockIdx.y, chunk = blockIdx.x;
    const int N = a.N, D = a.D;
    const int K = EXACT ? KB : a.K;
    const int KK = K * (K + 1) / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid >> 2, e = tid & 3;
    const int lane = tid & 31, gbase = lane & ~3;
    const int rr = e >> 1, cc = e & 1;
    const int KN4 = K * N * 4;

    unsigned char* stage = smem;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NST * stage_bytes);
    float2* Js = reinterpret_cast<float2*>(smem + NST * stage_bytes + BAR_BYTES);  // [K][N][4]
    float2* Es = Js + KN4;                                // [K][N][4] eta or x
    float2* acc = Es + KN4;                               // [K][N][4] first-station sums
    // Hessian pass: second-station sums in their own array, so the two scatter phases of a
    // diagonal need no barrier between them (the next diagonal's stage barrier orders them).
    float2* accs = HV ? acc + KN4 : acc;
    double* red = reinterpret_cast<double*>(accs + KN4);  // [64]

    {   // stage J and eta / x, clear the sums: 16-byte accesses (a station block is 32 bytes)
        const float4* Jg = reinterpret_cast<const float4*>(a.J) + (size_t)agent * KN4 / 2;
        const float4* Eg = reinterpret_cast<const float4*>(a.eta) + (size_t)agent * KN4 / 2;
        float4* J4 = reinterpret_cast<float4*>(Js);
        float4* E4 = reinterpret_cast<float4*>(Es);
        float4* A4 = reinterpret_cast<float4*>(acc);
        float4* S4 = reinterpret_cast<float4*>(accs);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = tid; i < KN4 / 2; i += nthr) {
            J4[i] = __ldg(Jg + i);
            E4[i] = __ldg(Eg + i);
            A4[i] = z4;
            if (HV) S4[i] = z4;
        }
    }
    const int d0 = 1 + chunk * a.chunk_diags;
    const int d1 = min(D, d0 + a.chunk_diags - 1);
    const int S = d1 >= d0 ? d1 - d0 + 1 : 0;  // one stage per diagonal
    const DiagDesc* dsc_agent = a.desc + (size_t)agent * D;

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int s2) {
        const DiagDesc d2 = dsc_agent[d0 + s2 - 1];
        const uint32_t ub = HV ? 0u : (uint32_t)(d2.n_pad * K * 32);
        const uint32_t sb = (uint32_t)(d2.n_pad * KK * 8);
        unsigned char* buf = stage + (s2 % NST) * stage_bytes;
        uint64_t* b = &bar[s2 % NST];
        mbar_expect_tx(b, ub + sb);
        if (ub) bulk_g2s(buf, a.U + d2.uoff, ub, b);
        if (sb) bulk_g2s(buf + ub, a.S + d2.soff, sb, b);
    };
    if (tid == 0)
        for (int s2 = 0; s2 < min(NST - 1, S); ++s2) issue(s2);

    double dcost = 0.0;
    for (int s = 0; s < S; ++s) {
        const DiagDesc dsc = dsc_agent[d0 + s - 1];
        __syncthreads();  // the buffer of stage s + NST - 1 is free
        if (tid == 0 && s + NST - 1 < S) {
            fence_proxy_async_smem();
            issue(s + NST - 1);
        }
        const bool ok = mbar_wait_bounded(&bar[s % NST], (uint32_t)((s / NST) & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(a.status, STATUS_TIMEOUT);
                const int last = min(S - 1, s + NST - 1);
                for (int s2 = s; s2 <= last; ++s2) mbar_wait_bounded(&bar[s2 % NST], (uint32_t)((s2 / NST) & 1));
            }
            return;
        }
        const unsigned char* buf = stage + (s % NST) * stage_bytes;
        const float2* Us = reinterpret_cast<const float2*>(buf);  // [n_pad][K][4] (trial)
        const float2* Ss = reinterpret_cast<const float2*>(buf + (HV ? 0 : dsc.n_pad * K * 32)) + (size_t)g * KK;
        const bool active = g < dsc.n;
        int first = 0, second = 0;
        float2 X[KB];  // station terms are -X_k J_s (first) and -X_k^H J_f (second)
#pragma unroll
        for (int k = 0; k < KB; ++k) X[k] = make_float2(0.f, 0.f);
        if (active) {
            const int sl = a.slot[dsc.slot_off + g];
            first = sl & 0xff;
            second = (sl >> 8) & 0xff;
            float2 Pa[KB], Pb[KB];  // Hessian: Q; trial: P and dP
#pragma unroll
            for (int l = 0; l < KB; ++l) {
                if (l < K) {
                    // row rr of J_f / eta_f and row cc of J_s / eta_s, one 16-byte load each
                    const float4 jf = *reinterpret_cast<const float4*>(Js + (l * N + first) * 4 + rr * 2);
                    const float4 js = *reinterpret_cast<const float4*>(Js + (l * N + second) * 4 + cc * 2);
                    const float4 ef = *reinterpret_cast<const float4*>(Es + (l * N + first) * 4 + rr * 2);
                    const float4 es = *reinterpret_cast<const float4*>(Es + (l * N + second) * 4 + cc * 2);
                    const float2 jf0 = make_float2(jf.x, jf.y), jf1 = make_float2(jf.z, jf.w);
                    const float2 js0 = make_float2(js.x, js.y), js1 = make_float2(js.z, js.w);
                    const float2 ef0 = make_float2(ef.x, ef.y), ef1 = make_float2(ef.z, ef.w);
                    const float2 es0 = make_float2(es.x, es.y), es1 = make_float2(es.z, es.w);
                    const float2 jfs = f2add(cmul_cb(jf0, js0), cmul_cb(jf1, js1));
                    const float2 efs = f2add(cmul_cb(ef0, js0), cmul_cb(ef1, js1));
                    const float2 jfe = f2add(cmul_cb(jf0, es0), cmul_cb(jf1, es1));
                    if (HV) {
                        Pa[l] = f2add(efs, jfe);
                    } else {
                        const float2 efe = f2add(cmul_cb(ef0, es0), cmul_cb(ef1, es1));
                        Pa[l] = jfs;
                        Pb[l] = f2add(f2add(efs, jfe), efe);
                    }
                } else {
                    Pa[l] = make_float2(0.f, 0.f);
                    Pb[l] = make_float2(0.f, 0.f);
                }
            }
            float dcf = 0.f;
            // small exact K: the packed S of the slot in registers, each entry loaded once
            constexpr bool SREG = EXACT && KB <= 6;
            constexpr int KKR = SREG ? KB * (KB + 1) / 2 : 1;
            float2 Sr[KKR];
            if (SREG) {
#pragma unroll
                for (int i = 0; i < KKR; ++i) Sr[i] = Ss[i];
            }
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k < K) {
                    float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
#pragma unroll
                    for (int l = 0; l < KB; ++l) {
                        if (l < K) {
                            // S_kl from the packed upper triangle; S_kl = conj(S_lk) below the diagonal
                            const int lo = k < l ? k : l, hi = k < l ? l : k;
                            const int si = lo * K - lo * (lo - 1) / 2 + (hi - lo);
                            float2 skl = SREG ? Sr[si < KKR ? si : 0] : Ss[si];
                            if (k > l) skl.y = -skl.y;
                            cmac(sa, skl, Pa[l]);
                            if (!HV) cmac(sb, skl, Pb[l]);
                        }
                    }
                    if (HV) {
                        X[k] = make_float2(-sa.x, -sa.y);  // X = -(S Q)_k
                    } else {
                        const float2 W = f2sub(Us[((size_t)g * K + k) * 4 + e], sa);  // W_k at J
                        // decrease: Re[conj(dP_k) (2 W_k - (S dP)_k)]
                        const float2 t = make_float2(2.f * W.x - sb.x, 2.f * W.y - sb.y);
                        dcf = fmaf(Pb[k].x, t.x, fmaf(Pb[k].y, t.y, dcf));
                        X[k] = f2sub(W, sb);  // W'_k at J' = J + x
                    }
                }
            }
            dcost += (double)dcf;
        }
        // Phase 1: first station receives -X_k J'_s (J' = J + x in the trial pass).
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k < K) {
                const float2 w0 = shfl2(X[k], gbase + rr * 2 + 0);
                const float2 w1 = shfl2(X[k], gbase + rr * 2 + 1);
                if (active) {
                    const float2* js = Js + (k * N + second) * 4;
                    float2 j0 = js[0 * 2 + cc], j1 = js[1 * 2 + cc];
                    if (!HV) {
                        const float2* xs = Es + (k * N + second) * 4;
                        j0 = f2add(j0, xs[0 * 2 + cc]);
                        j1 = f2add(j1, xs[1 * 2 + cc]);
                    }
                    const float2 v = f2add(cmul(w0, j0), cmul(w1, j1));
                    float2* dd = acc + (k * N + first) * 4 + e;
                    *dd = f2sub(*dd, v);
                }
            }
        }
        if (!HV) __syncthreads();
        // Phase 2: second station receives -X_k^H J'_f.
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            if (k < K) {
                const float2 w0 = shfl2(X[k], gbase + 0 * 2 + rr);
                const float2 w1 = shfl2(X[k], gbase + 1 * 2 + rr);
                if (active) {
                    const float2* jf = Js + (k * N + first) * 4;
                    float2 j0 = jf[0 * 2 + cc], j1 = jf[1 * 2 + cc];
                    if (!HV) {
                        const float2* xf = Es + (k * N + first) * 4;
                        j0 = f2add(j0, xf[0 * 2 + cc]);
                        j1 = f2add(j1, xf[1 * 2 + cc]);
                    }
                    const float2 v = f2add(cmul_ca(w0, j0), cmul_ca(w1, j1));
                    float2* dd = accs + (k * N + second) * 4 + e;
                    *dd = f2sub(*dd, v);
                }
            }
        }
    }
    __syncthreads();
    float4* out = reinterpret_cast<float4*>(a.part) + ((size_t)agent * a.n_chunks + chunk) * KN4 / 2;
    for (int i = tid; i < KN4 / 2; i += nthr) {
        float4 v = reinterpret_cast<const float4*>(acc)[i];
        if (HV) {
            const float4 w = reinterpret_cast<const float4*>(accs)[i];
            v = make_float4(v.x + w.x, v.y + w.y, v.z + w.z, v.w + w.w);
        }
        out[i] = v;
    }
    if (!HV) {
        for (int o = 16; o > 0; o >>= 1) dcost += __shfl_down_sync(0xffffffffu, dcost, o);
        if (lane == 0) red[tid >> 5] = dcost;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (nthr >> 5); ++w) s += red[w];
            a.part_dcost[(size_t)agent * a.n_chunks + chunk] = s;
        }
    }
}

template <int KB, bool HV>
cudaError_t prep_kb() {
    cudaError_t e = cudaFuncSetAttribute(k_ss_sweep<KB, HV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_ss_sweep<KB, HV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <bool HV>
cudaError_t prep_all() {
    cudaError_t e;
    if ((e = prep_kb<1, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<2, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<3, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<4, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<5, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<6, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<8, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<10, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<12, HV>()) != cudaSuccess) return e;
    return prep_kb<16, HV>();
}

template <int KB, bool HV>
cudaError_t go(const SSArgs& a, int threads, size_t smem, int sb, cudaStream_t s) {
    if (a.K == KB)
        k_ss_sweep<KB, HV, true><<<dim3(a.n_chunks, a.A), threads, smem, s>>>(a, sb);
    else
        k_ss_sweep<KB, HV, false><<<dim3(a.n_chunks, a.A), threads, smem, s>>>(a, sb);
    return cudaGetLastError();
}

template <bool HV>
cudaError_t dispatch(const SSArgs& a, int threads, size_t smem, int sb, cudaStream_t s) {
    const int K = a.K;
    if (K <= 1) return go<1, HV>(a, threads, smem, sb, s);
    if (K <= 2) return go<2, HV>(a, threads, smem, sb, s);
    if (K <= 3) return go<3, HV>(a, threads, smem, sb, s);
    if (K <= 4) return go<4, HV>(a, threads, smem, sb, s);
    if (K <= 5) return go<5, HV>(a, threads, smem, sb, s);
    if (K <= 6) return go<6, HV>(a, threads, smem, sb, s);
    if (K <= 8) return go<8, HV>(a, threads, smem, sb, s);
    if (K <= 10) return go<10, HV>(a, threads, smem, sb, s);
    if (K <= 12) return go<12, HV>(a, threads, smem, sb, s);
    return go<16, HV>(a, threads, smem, sb, s);
}

}  // namespace

cudaError_t prepare_ss_kernels() {
    cudaError_t e = prep_all<false>();
    return e != cudaSuccess ? e : prep_all<true>();
}

cudaError_t launch_ss_sweep(const SSArgs& a, bool hessvec, cudaStream_t s) {
    const int KK = a.K * (a.K + 1) / 2;
    const int per_slot = (hessvec ? 0 : a.K * 32) + KK * 8;
    const int sb = ((a.slots_max * per_slot + 127) / 128) * 128;
    const size_t smem = (size_t)NST * sb + BAR_BYTES + (size_t)(hessvec ? 4 : 3) * a.K * a.N * 32 + 64 * 8;
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    const int threads = ((4 * a.slots_max + 31) / 32) * 32;
    return hessvec ? dispatch<true>(a, threads, smem, sb, s) : dispatch<false>(a, threads, smem, sb, s);
}

}  // namespace calib
