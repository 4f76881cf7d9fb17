// Baseline sweeps of the J-update (Section 3, Eq. M1): one pass over an agent's baselines
// and samples that either
//   (residual pass)  forms R_t = V_t - sum_k c_tk J_pk J_qk^H, the data cost sum ||R_t||^2 and
//                    the station sums of grad g (Section 3, the expression for grad_i(g)):
//                    station p gets -sum_t conj(c_tk) R_t J_qk, station q gets -sum_t c_tk R_t^H J_pk;
//   (Hessian pass)   forms dM_t = sum_k c_tk (eta_pk J_qk^H + J_pk eta_qk^H) and the station sums of
//                    the Gauss-Newton Hessian-vector product: p gets sum_t conj(c_tk) dM_t J_qk,
//                    q gets sum_t c_tk dM_t^H J_pk (Eq. HessL, GN part of Hess g).
//   (trial pass)     the residual pass at J' = J + x that also returns the decrease of the data cost
//                    g(J) - g(J') = sum_t Re[(2 R_t - dM_t)^H dM_t], dM_t = sum_k c_tk (x_pk J_qk^H +
//                    J_pk x_qk^H + x_pk x_qk^H). Formed from the small dM_t it is accurate relative to the
//                    decrease itself, which a difference of two float32 costs is not near convergence.
// All use W_k = sum_t conj(c_tk) X_t with X_t = R_t (residual, trial) or -dM_t (Hessian), so the
// station terms are -W_k J_qk and -W_k^H J_pk in every mode (J' in place of J for the trial pass).
//
// Mapping: one CTA per (agent, chunk of circulant diagonals); four threads per baseline slot,
// one per correlation (element (r,c) of the 2x2 block). Within a diagonal each station is the
// first element of at most one slot and the second of at most one, so the station sums are
// accumulated in shared memory in two barrier-separated phases without atomics: the order of
// every addition is fixed, and the result is bitwise reproducible.
// Data tiles (all slots of one diagonal, TT samples) are streamed from HBM into a 3-stage
// shared-memory ring with cp.async.bulk (TMA bulk copies) completing on mbarriers; every wait
// is bounded and reports a timeout through the status word instead of hanging.
#include "calib_internal.cuh"
#include "tma.cuh"

namespace calib {
namespace {

constexpr int NST = 3;


__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmul_cb(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
__device__ __forceinline__ float2 cmul_ca(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

enum { M_RESID = 0, M_HV = 1, M_TRIAL = 2 };

// KB: register bucket; EXACT: K == KB, so loop bounds and strides over K are constants.
template <int KB, int MODE, bool EXACT>
__global__ void __launch_bounds__(512) k_sweep(const SweepArgs a, const int stage_bytes) {
    constexpr bool HV = MODE == M_HV;
    constexpr bool TR = MODE == M_TRIAL;
    extern __shared__ __align__(128) unsigned char smem[];
    const int agent = blockIdx.y;
    const int chunk = blockIdx.x;
    const int N = a.N, D = a.D;
    const int K = EXACT ? KB : a.K;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid >> 2, e = tid & 3;
    const int lane = tid & 31, gbase = lane & ~3;
    const int rr = e >> 1, cc = e & 1;
    const int KN4 = K * N * 4;

    unsigned char* stage = smem;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NST * stage_bytes);
    float2* Js = reinterpret_cast<float2*>(bar + NST);  // [K][N][4]
    float2* Es = Js + KN4;                                // [K][N][4] direction (Hessian) / step x (trial)
    float2* acc = (HV || TR) ? (Es + KN4) : Es;           // [K][N][4] station sums
    double* red = reinterpret_cast<double*>(acc + KN4);   // [64]

    const float2* Jg = reinterpret_cast<const float2*>(a.J) + (size_t)agent * KN4;
    for (int i = tid; i < KN4; i += nthr) Js[i] = Jg[i];
    if (HV || TR) {
        const float2* Eg = reinterpret_cast<const float2*>(a.eta) + (size_t)agent * KN4;
        for (int i = tid; i < KN4; i += nthr) Es[i] = Eg[i];
    }
    for (int i = tid; i < KN4; i += nthr) acc[i] = make_float2(0.f, 0.f);

    const int Ta = a.T[agent];
    const int d0 = 1 + chunk * a.chunk_diags;
    const int d1 = min(D, d0 + a.chunk_diags - 1);
    const int ndiag = d1 >= d0 ? d1 - d0 + 1 : 0;
    const int ntile = (Ta + a.TT - 1) / a.TT;
    const int S = ndiag * ntile;
    const DiagDesc* dsc_agent = a.desc + (size_t)agent * D;

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int s2) {
        const int di2 = s2 / ntile, tile2 = s2 - di2 * ntile;
        const DiagDesc d2 = dsc_agent[d0 + di2 - 1];
        const int t0 = tile2 * a.TT, nt = min(a.TT, Ta - t0);
        const uint32_t vb = HV ? 0u : (uint32_t)(nt * d2.n_pad * 32);
        const uint32_t cb = (uint32_t)(nt * d2.n_pad * K * 8);
        unsigned char* buf = stage + (s2 % NST) * stage_bytes;
        uint64_t* b = &bar[s2 % NST];
        mbar_expect_tx(b, vb + cb);
        if (vb) bulk_g2s(buf, a.V + d2.voff + (size_t)t0 * d2.n_pad * 4, vb, b);
        if (cb) bulk_g2s(buf + vb, a.C + d2.coff + (size_t)t0 * d2.n_pad * K, cb, b);
    };
    if (tid == 0) {
        for (int s2 = 0; s2 < min(NST - 1, S); ++s2) issue(s2);
    }

    float2 P[KB], W[KB], DP[TR ? KB : 1];
#pragma unroll
    for (int k = 0; k < KB; ++k) { P[k] = make_float2(0.f, 0.f); W[k] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int k = 0; k < (TR ? KB : 1); ++k) DP[k] = make_float2(0.f, 0.f);
    bool active = false;
    int first = 0, second = 0;
    double cost = 0.0, dcost = 0.0;

    for (int s = 0; s < S; ++s) {
        const int di = s / ntile, tile = s - di * ntile;
        const DiagDesc dsc = dsc_agent[d0 + di - 1];
        if (tile == 0) {
            active = g < dsc.n;
            if (active) {
                const int sl = a.slot[dsc.slot_off + g];
                first = sl & 0xff;
                second = (sl >> 8) & 0xff;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k < K) {
                        const float2* jf = Js + (k * N + first) * 4;
                        const float2* js = Js + (k * N + second) * 4;
                        // P_k[rr][cc] = sum_m J_f[rr][m] conj(J_s[cc][m])
                        float2 v = f2add(cmul_cb(jf[rr * 2 + 0], js[cc * 2 + 0]), cmul_cb(jf[rr * 2 + 1], js[cc * 2 + 1]));
                        if (HV || TR) {
                            const float2* ef = Es + (k * N + first) * 4;
                            const float2* es = Es + (k * N + second) * 4;
                            // Q_k = eta_f J_s^H + J_f eta_s^H
                            float2 q = f2add(f2add(cmul_cb(ef[rr * 2 + 0], js[cc * 2 + 0]), cmul_cb(ef[rr * 2 + 1], js[cc * 2 + 1])),
                                             f2add(cmul_cb(jf[rr * 2 + 0], es[cc * 2 + 0]), cmul_cb(jf[rr * 2 + 1], es[cc * 2 + 1])));
                            if (TR) {  // + x_f x_s^H: the exact change of J_f J_s^H
                                q = f2add(q, f2add(cmul_cb(ef[rr * 2 + 0], es[cc * 2 + 0]), cmul_cb(ef[rr * 2 + 1], es[cc * 2 + 1])));
                                DP[TR ? k : 0] = q;
                            } else {
                                v = q;
                            }
                        }
                        P[k] = v;
                        W[k] = make_float2(0.f, 0.f);
                    }
                }
            }
        }
        __syncthreads();  // every thread is done with the buffer that stage s + NST - 1 reuses
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

        const int t0 = tile * a.TT, nt = min(a.TT, Ta - t0);
        const unsigned char* buf = stage + (s % NST) * stage_bytes;
        const float2* Vs = reinterpret_cast<const float2*>(buf);
        const float2* Cs = reinterpret_cast<const float2*>(buf + (HV ? 0 : nt * dsc.n_pad * 32));
        if (active) {
            float costf = 0.f, dcostf = 0.f;
            for (int tl = 0; tl < nt; ++tl) {
                const float2* cp = Cs + (size_t)(tl * dsc.n_pad + g) * K;
                float2 cv[KB];
                float mr = 0.f, mi = 0.f, dr = 0.f, di = 0.f;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k < K) {
                        cv[k] = cp[k];
                        mr = fmaf(cv[k].x, P[k].x, fmaf(-cv[k].y, P[k].y, mr));
                        mi = fmaf(cv[k].x, P[k].y, fmaf(cv[k].y, P[k].x, mi));
                        if (TR) {
                            const float2 q = DP[TR ? k : 0];
                            dr = fmaf(cv[k].x, q.x, fmaf(-cv[k].y, q.y, dr));
                            di = fmaf(cv[k].x, q.y, fmaf(cv[k].y, q.x, di));
                        }
                    }
                }
                float xr, xi;
                if (!HV) {
                    const float2 v = Vs[(tl * dsc.n_pad + g) * 4 + e];
                    xr = v.x - mr;
                    xi = v.y - mi;
                    if (TR) {  // decrease |R|^2 - |R - dM|^2 = (2R - dM) . dM, then R <- R - dM
                        dcostf = fmaf(2.f * xr - dr, dr, fmaf(2.f * xi - di, di, dcostf));
                        xr -= dr;
                        xi -= di;
                    }
                    costf = fmaf(xr, xr, fmaf(xi, xi, costf));
                } else {
                    xr = -mr;
                    xi = -mi;
                }
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k < K) {  // W_k += conj(c) X
                        W[k].x = fmaf(cv[k].x, xr, fmaf(cv[k].y, xi, W[k].x));
                        W[k].y = fmaf(cv[k].x, xi, fmaf(-cv[k].y, xr, W[k].y));
                    }
                }
            }
            cost += (double)costf;
            dcost += (double)dcostf;
        }

        if (tile == ntile - 1) {
            // Phase 1: first station of each slot receives -W_k J_sk (row rr of W times column cc of J_s).
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k < K) {
                    const float2 w0 = shfl2(W[k], gbase + rr * 2 + 0);
                    const float2 w1 = shfl2(W[k], gbase + rr * 2 + 1);
                    if (active) {
                        const float2* js = Js + (k * N + second) * 4;
                        float2 j0 = js[0 * 2 + cc], j1 = js[1 * 2 + cc];
                        if (TR) {
                            const float2* xs = Es + (k * N + second) * 4;
                            j0 = f2add(j0, xs[0 * 2 + cc]);
                            j1 = f2add(j1, xs[1 * 2 + cc]);
                        }
                        const float2 v = f2add(cmul(w0, j0), cmul(w1, j1));
                        float2* d = acc + (k * N + first) * 4 + e;
                        *d = make_float2(d->x - v.x, d->y - v.y);
                    }
                }
            }
            __syncthreads();
            // Phase 2: second station receives -W_k^H J_fk.
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k < K) {
                    const float2 w0 = shfl2(W[k], gbase + 0 * 2 + rr);
                    const float2 w1 = shfl2(W[k], gbase + 1 * 2 + rr);
                    if (active) {
                        const float2* jf = Js + (k * N + first) * 4;
                        float2 j0 = jf[0 * 2 + cc], j1 = jf[1 * 2 + cc];
                        if (TR) {
                            const float2* xf = Es + (k * N + first) * 4;
                            j0 = f2add(j0, xf[0 * 2 + cc]);
                            j1 = f2add(j1, xf[1 * 2 + cc]);
                        }
                        const float2 v = f2add(cmul_ca(w0, j0), cmul_ca(w1, j1));
                        float2* d = acc + (k * N + second) * 4 + e;
                        *d = make_float2(d->x - v.x, d->y - v.y);
                    }
                }
            }
        }
    }
    __syncthreads();

    float2* out = reinterpret_cast<float2*>(a.part) + ((size_t)agent * a.n_chunks + chunk) * KN4;
    for (int i = tid; i < KN4; i += nthr) out[i] = acc[i];
    if (!HV) {
        for (int o = 16; o > 0; o >>= 1) {
            cost += __shfl_down_sync(0xffffffffu, cost, o);
            if (TR) dcost += __shfl_down_sync(0xffffffffu, dcost, o);
        }
        if (lane == 0) {
            red[tid >> 5] = cost;
            red[32 + (tid >> 5)] = dcost;
        }
        __syncthreads();
        if (tid == 0) {
            double s = 0.0, ds = 0.0;
            for (int w = 0; w < (nthr >> 5); ++w) {
                s += red[w];
                ds += red[32 + w];
            }
            a.part_cost[(size_t)agent * a.n_chunks + chunk] = s;
            if (TR) a.part_dcost[(size_t)agent * a.n_chunks + chunk] = ds;
        }
    }
}

template <int KB, int HV>
cudaError_t prepare_kb() {
    cudaError_t e = cudaFuncSetAttribute(k_sweep<KB, HV, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sweep<KB, HV, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

template <int KB, int HV>
cudaError_t launch_kb(const SweepArgs& a, int threads, size_t smem, int stage_bytes, cudaStream_t s) {
    dim3 grid(a.n_chunks, a.A);
    if (a.K == KB)
        k_sweep<KB, HV, true><<<grid, threads, smem, s>>>(a, stage_bytes);
    else
        k_sweep<KB, HV, false><<<grid, threads, smem, s>>>(a, stage_bytes);
    return cudaGetLastError();
}

template <int HV>
cudaError_t dispatch(const SweepArgs& a, int threads, size_t smem, int stage_bytes, cudaStream_t s) {
    switch (a.K <= 1 ? 1 : a.K <= 2 ? 2 : a.K <= 3 ? 3 : a.K <= 4 ? 4 : a.K <= 5 ? 5 : a.K <= 6 ? 6
            : a.K <= 8 ? 8 : a.K <= 10 ? 10 : a.K <= 12 ? 12 : 16) {
        case 1: return launch_kb<1, HV>(a, threads, smem, stage_bytes, s);
        case 2: return launch_kb<2, HV>(a, threads, smem, stage_bytes, s);
        case 3: return launch_kb<3, HV>(a, threads, smem, stage_bytes, s);
        case 4: return launch_kb<4, HV>(a, threads, smem, stage_bytes, s);
        case 5: return launch_kb<5, HV>(a, threads, smem, stage_bytes, s);
        case 6: return launch_kb<6, HV>(a, threads, smem, stage_bytes, s);
        case 8: return launch_kb<8, HV>(a, threads, smem, stage_bytes, s);
        case 10: return launch_kb<10, HV>(a, threads, smem, stage_bytes, s);
        case 12: return launch_kb<12, HV>(a, threads, smem, stage_bytes, s);
        default: return launch_kb<16, HV>(a, threads, smem, stage_bytes, s);
    }
}

int stage_bytes_for(int slots_max, int K, bool hessvec, int TT) {
    const int per_t = slots_max * (hessvec ? 8 * K : 32 + 8 * K);
    return ((TT * per_t + 127) / 128) * 128;
}

template <int HV>
cudaError_t prepare_all() {
    cudaError_t e;
    if ((e = prepare_kb<1, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<2, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<3, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<4, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<5, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<6, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<8, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<10, HV>()) != cudaSuccess) return e;
    if ((e = prepare_kb<12, HV>()) != cudaSuccess) return e;
    return prepare_kb<16, HV>();
}

}  // namespace

cudaError_t prepare_sweep_kernels() {
    cudaError_t e = prepare_all<M_RESID>();
    if (e == cudaSuccess) e = prepare_all<M_HV>();
    return e != cudaSuccess ? e : prepare_all<M_TRIAL>();
}

int sweep_threads(int slots_max) { return ((4 * slots_max + 31) / 32) * 32; }

int sweep_tile_samples(int slots_max, int K, bool hessvec) {
    const int per_t = slots_max * (hessvec ? 8 * K : 32 + 8 * K);
    int tt = (24 * 1024) / (per_t > 0 ? per_t : 1);
    return tt < 1 ? 1 : tt;
}

size_t sweep_smem_bytes(int N, int K, bool two_vectors) {
    // stage ring is sized per launch; this is the fixed part (barriers, J, eta or x, sums, scratch)
    return (size_t)NST * 8 + (size_t)(two_vectors ? 3 : 2) * K * N * 32 + 64 * 8;
}

cudaError_t launch_sweep(const SweepArgs& a, int mode, cudaStream_t s) {
    const bool hessvec = mode == SWEEP_HESSVEC;
    const int threads = sweep_threads(a.slots_max);
    const int sb = stage_bytes_for(a.slots_max, a.K, hessvec, a.TT);
    const size_t smem = (size_t)NST * sb + sweep_smem_bytes(a.N, a.K, mode != SWEEP_RESIDUAL);
    if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
    if (mode == SWEEP_HESSVEC) return dispatch<M_HV>(a, threads, smem, sb, s);
    if (mode == SWEEP_TRIAL) return dispatch<M_TRIAL>(a, threads, smem, sb, s);
    return dispatch<M_RESID>(a, threads, smem, sb, s);
}

}  // namespace calib
