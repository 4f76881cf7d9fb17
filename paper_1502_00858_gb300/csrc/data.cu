// Data ingestion and coherency prediction.
//
// Ingestion moves user-layout visibilities [A][B][T_a][2][2] and coherencies [A][B][T_a][K] into
// the circulant-diagonal layout used by the sweeps (see calib_internal.cuh); a pair held reversed
// gets V^H and conj(c), which is the same measurement seen from the other station (Eq. vispq).
//
// Prediction (Eq. coh): c_pq = sum_s I_s(f) exp(i phi_pq,s) with phi = -2 pi (f/c)
// (u_pq l + v_pq m + w_pq (n - 1)) and (u,v,w)_pq = (u,v,w)_p - (u,v,w)_q. The phase splits into
// station phasors E_ps = exp(-2 pi i turns_ps), turns_ps = (f/c)(u_p l + v_p m + w_p (n-1)), so
// c_pq = sum_s I_s E_ps conj(E_qs). Turns are formed in float64 and reduced to [-1/2, 1/2]
// before the float32 sincospi, so the phase error does not grow with baseline length.
#include <math.h>

#include <algorithm>

#include "calib_internal.cuh"
#include "tma.cuh"

namespace calib {
namespace {

constexpr double C_LIGHT = 299792458.0;

__global__ void k_ingest(const IngestArgs a) {
    const int d = blockIdx.x, agent = blockIdx.y;
    const DiagDesc dsc = a.desc[(size_t)agent * a.D + d];
    const int Ta = a.T[agent];
    const int w = a.is_vis ? 4 : a.K;
    const long long total = (long long)Ta * dsc.n_pad * w;
    float2* dst = a.dst + (a.is_vis ? dsc.voff : dsc.coff);
    const float2* src = a.src + a.src_off[agent];
    for (long long i = threadIdx.x; i < total; i += blockDim.x) {
        const int e = (int)(i % w);
        const long long rest = i / w;
        const int g = (int)(rest % dsc.n_pad);
        const int t = (int)(rest / dsc.n_pad);
        float2 v = make_float2(0.f, 0.f);
        if (g < dsc.n) {
            const int sl = a.slot[dsc.slot_off + g];
            const int rev = (sl >> 16) & 1;
            const long long b = a.slot_b[dsc.slot_off + g];
            if (a.is_vis) {
                const int es = rev ? ((e & 1) * 2 + (e >> 1)) : e;  // V^H: element (r,c) <- conj (c,r)
                v = src[(b * Ta + t) * 4 + es];
            } else {
                v = src[(b * Ta + t) * a.K + e];
            }
            if (rev) v.y = -v.y;
        }
        dst[i] = v;
    }
}

__global__ void k_extract_coh(const IngestArgs a, float2* out) {
    const int d = blockIdx.x, agent = blockIdx.y;
    const DiagDesc dsc = a.desc[(size_t)agent * a.D + d];
    const int Ta = a.T[agent];
    const long long total = (long long)Ta * dsc.n * a.K;
    const float2* src = a.dst + dsc.coff;
    float2* o = out + a.src_off[agent];
    for (long long i = threadIdx.x; i < total; i += blockDim.x) {
        const int k = (int)(i % a.K);
        const long long rest = i / a.K;
        const int g = (int)(rest % dsc.n);
        const int t = (int)(rest / dsc.n);
        const int sl = a.slot[dsc.slot_off + g];
        const long long b = a.slot_b[dsc.slot_off + g];
        float2 v = src[((long long)t * dsc.n_pad + g) * a.K + k];
        if ((sl >> 16) & 1) v.y = -v.y;
        o[(b * Ta + t) * a.K + k] = v;
    }
}

// Residual visibilities (Section 2: the solutions correct the data, and the residual is the data
// minus the predicted model). In the layout's station order (i, j), where the data are V_ij and the
// coherencies c_ij: R = V_ij - sum_{k in mask} c_ij,k J_ik J_jk^H, then, with a correction
// direction k0, R <- J_i,k0^-1 R J_j,k0^-H. A pair held reversed is written back as R^H, which is
// the user-order residual (and correction) of the same baseline. One CTA per (diagonal, agent), one
// thread per slot looping over the samples; reads V and C once and writes each residual once.
// Each M_k = J_ik J_jk^H is formed once per slot (below), not once per sample.
struct cf { float x, y; };
__device__ __forceinline__ cf cmulf(cf a, cf b) { return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cf cmulcf(cf a, cf b) { return cf{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }  // conj(a) b
__device__ __forceinline__ cf caddf(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
struct m22 { cf e[2][2]; };
__device__ __forceinline__ m22 ld_m22(const float4* rows) {
    const float4 r0 = __ldg(rows), r1 = __ldg(rows + 1);
    return m22{{{cf{r0.x, r0.y}, cf{r0.z, r0.w}}, {cf{r1.x, r1.y}, cf{r1.z, r1.w}}}};
}
// A B
__device__ __forceinline__ m22 mmul(const m22& A, const m22& B) {
    m22 o;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) o.e[r][c] = caddf(cmulf(A.e[r][0], B.e[0][c]), cmulf(A.e[r][1], B.e[1][c]));
    return o;
}
// A^-1 by the adjugate: [[a11, -a01], [-a10, a00]] / (a00 a11 - a01 a10)
__device__ __forceinline__ m22 minv(const m22& A) {
    const cf a = cmulf(A.e[0][0], A.e[1][1]), b = cmulf(A.e[0][1], A.e[1][0]);
    const cf det{a.x - b.x, a.y - b.y};
    const float s = 1.f / (det.x * det.x + det.y * det.y);
    const cf id{det.x * s, -det.y * s};  // 1 / det
    m22 o;
    o.e[0][0] = cmulf(A.e[1][1], id);
    o.e[1][1] = cmulf(A.e[0][0], id);
    o.e[0][1] = cmulf(cf{-A.e[0][1].x, -A.e[0][1].y}, id);
    o.e[1][0] = cmulf(cf{-A.e[1][0].x, -A.e[1][0].y}, id);
    return o;
}
__device__ __forceinline__ m22 mherm(const m22& A) {
    m22 o;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) o.e[r][c] = cf{A.e[c][r].x, -A.e[c][r].y};
    return o;
}

constexpr int RES_THREADS = 64;

// Before its sample loop a thread forms its slot's model matrices M_k = J_ik J_jk^H of the masked
// directions into its own column of shared memory (Ms: [K][2 rows][RES_THREADS] float4; no thread
// reads another's), so the loop over the samples reads only V, C and M.
__global__ void __launch_bounds__(RES_THREADS) k_residual(const ResidualArgs a) {
    extern __shared__ float4 Ms[];
    const int d = blockIdx.x, agent = blockIdx.y, tid = threadIdx.x;
    const DiagDesc dsc = a.desc[(size_t)agent * a.D + d];
    const int Ta = a.T[agent], K = a.K, N = a.N;
    const float4* __restrict__ J = reinterpret_cast<const float4*>(a.J) + (size_t)agent * K * N * 2;  // [K][N][2 rows]
    const float4* __restrict__ V = reinterpret_cast<const float4*>(a.V + dsc.voff);                 // [T][n_pad][2 rows]
    const float2* __restrict__ C = a.C + dsc.coff;                                                   // [T][n_pad][K]
    float4* __restrict__ out = reinterpret_cast<float4*>(a.out + a.vis_off[agent]);                 // [B][T_a][2 rows]
    for (int g = tid; g < dsc.n; g += RES_THREADS) {
        const int sl = a.slot[dsc.slot_off + g];
        const int i = sl & 0xff, j = (sl >> 8) & 0xff, rev = (sl >> 16) & 1;
        const long long b = a.slot_b[dsc.slot_off + g];
        m22 Li{}, Rj{};
        if (a.correct >= 0) {
            Li = minv(ld_m22(J + ((size_t)a.correct * N + i) * 2));
            Rj = mherm(minv(ld_m22(J + ((size_t)a.correct * N + j) * 2)));
        }
        for (int k = 0; k < K; ++k) {
            if (!((a.mask >> k) & 1u)) continue;
            const m22 Ji = ld_m22(J + ((size_t)k * N + i) * 2), Jj = ld_m22(J + ((size_t)k * N + j) * 2);
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                // (J_i J_j^H)[r][cc] = J_i[r][0] conj(J_j[cc][0]) + J_i[r][1] conj(J_j[cc][1])
                const cf m0 = caddf(cmulcf(Jj.e[0][0], Ji.e[r][0]), cmulcf(Jj.e[0][1], Ji.e[r][1]));
                const cf m1 = caddf(cmulcf(Jj.e[1][0], Ji.e[r][0]), cmulcf(Jj.e[1][1], Ji.e[r][1]));
                Ms[(k * 2 + r) * RES_THREADS + tid] = make_float4(m0.x, m0.y, m1.x, m1.y);
            }
        }
#pragma unroll 2
        for (int t = 0; t < Ta; ++t) {
            const size_t pos = (size_t)t * dsc.n_pad + g;
            m22 R = ld_m22(V + pos * 2);
            for (int k = 0; k < K; ++k) {
                if (!((a.mask >> k) & 1u)) continue;
                const float2 c2 = __ldg(C + pos * K + k);
                const cf c{c2.x, c2.y};
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4 q = Ms[(k * 2 + r) * RES_THREADS + tid];
                    const cf m[2] = {cf{q.x, q.y}, cf{q.z, q.w}};
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        const cf cm = cmulf(c, m[cc]);
                        R.e[r][cc] = cf{R.e[r][cc].x - cm.x, R.e[r][cc].y - cm.y};
                    }
                }
            }
            if (a.correct >= 0) R = mmul(mmul(Li, R), Rj);
            if (rev) R = mherm(R);
            float4* o = out + ((size_t)b * Ta + t) * 2;
            o[0] = make_float4(R.e[0][0].x, R.e[0][0].y, R.e[0][1].x, R.e[0][1].y);
            o[1] = make_float4(R.e[1][0].x, R.e[1][0].y, R.e[1][1].x, R.e[1][1].y);
        }
    }
}

// One CTA per (sample, agent); source chunks sized to fit the phasor table in shared memory.
__global__ void __launch_bounds__(256) k_predict(const PredictArgs a, int s_chunk) {
    extern __shared__ __align__(128) unsigned char smem[];  // one declaration for the file's kernels
    const int t = blockIdx.x, agent = blockIdx.y;
    const int Ta = a.T[agent];
    if (t >= Ta) return;
    const int iv = agent / a.P, fi = agent - iv * a.P;
    const double f = a.freqs[fi];
    const int N = a.N, K = a.K;
    double* lmn = reinterpret_cast<double*>(smem);                        // [K][s_chunk][3] l, m, n - 1
    float2* E = reinterpret_cast<float2*>(lmn + (size_t)K * s_chunk * 3);  // [K][s_chunk][N]
    float* flux = reinterpret_cast<float*>(E + (size_t)K * s_chunk * N);  // [K][s_chunk]
    const double* uvw = a.uvw + (((size_t)iv * a.Tmax + t) * N) * 3;
    const DiagDesc* dsc_agent = a.desc + (size_t)agent * a.D;

    for (int s0 = 0; s0 < a.S; s0 += s_chunk) {
        const int ns = min(s_chunk, a.S - s0);
        // per source: flux at f and its direction (l, m, n - 1), scaled by f / c
        const double fc = f / C_LIGHT;
        for (int i = threadIdx.x; i < K * ns; i += blockDim.x) {
            const int k = i / ns, s = i - k * ns;
            const double* src = a.sky + ((size_t)k * a.S + s0 + s) * 4;
            flux[k * s_chunk + s] = (float)(src[2] * pow(f / a.f0, src[3]));
            const double l = src[0], m = src[1];
            const double r2 = l * l + m * m;
            double* d = lmn + ((size_t)k * s_chunk + s) * 3;
            d[0] = fc * l;
            d[1] = fc * m;
            d[2] = fc * (-r2 / (1.0 + sqrt(1.0 - r2)));  // sqrt(1 - l^2 - m^2) - 1, cancellation-free
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K * ns * N; i += blockDim.x) {
            const int p = i % N;
            const int ks = i / N;
            const int k = ks / ns, s = ks - k * ns;
            const double* d = lmn + ((size_t)k * s_chunk + s) * 3;
            const double turns = uvw[p * 3 + 0] * d[0] + uvw[p * 3 + 1] * d[1] + uvw[p * 3 + 2] * d[2];
            const float fr = (float)(turns - rint(turns));
            float sn, cs;
            sincospif(2.0f * fr, &sn, &cs);
            E[((size_t)k * s_chunk + s) * N + p] = make_float2(cs, -sn);  // exp(-2 pi i turns)
        }
        __syncthreads();
        for (int d = 0; d < a.D; ++d) {
            const DiagDesc dsc = dsc_agent[d];
            float2* out = a.C + dsc.coff + (size_t)t * dsc.n_pad * K;
            for (int it = threadIdx.x; it < dsc.n_pad * K; it += blockDim.x) {
                const int g = it / K, k = it - g * K;
                float2 c = make_float2(0.f, 0.f);
                if (g < dsc.n) {
                    const int sl = a.slot[dsc.slot_off + g];
                    const int p = sl & 0xff, q = (sl >> 8) & 0xff;
                    const float2* Ek = E + (size_t)k * s_chunk * N;
                    const float* fk = flux + k * s_chunk;
                    for (int s = 0; s < ns; ++s) {
                        const float2 ep = Ek[s * N + p], eq = Ek[s * N + q];
                        // I_s E_p conj(E_q)
                        const float re = ep.x * eq.x + ep.y * eq.y;
                        const float im = ep.y * eq.x - ep.x * eq.y;
                        c.x = fmaf(fk[s], re, c.x);
                        c.y = fmaf(fk[s], im, c.y);
                    }
                }
                if (s0 == 0) {
                    out[it] = c;
                } else {
                    const float2 o = out[it];
                    out[it] = make_float2(o.x + c.x, o.y + c.y);
                }
            }
        }
        __syncthreads();
    }
}

// Jacobi weights of one agent: gw[k][o][p] = gw[k][p][o] = s_bk = sum_t |c_btk|^2 for the baseline
// b = (p, o), zero for flagged baselines and o = p (fixed for the whole calibration). Each entry is
// written by the one slot that holds its station pair: no atomics.
// One CTA per (diagonal, agent); the entries no slot writes (the diagonal p = o, flagged pairs,
// the row padding) are zeroed by the launcher first.
__global__ void k_gram_weights(const float2* C, const DiagDesc* desc, const int* slot, const int* T, float* gw,
                               int D, int K, int N) {
    const int d = blockIdx.x, agent = blockIdx.y;
    const int NW = (N + 3) / 4 * 4;  // row stride: 16-byte rows
    float* W = gw + (size_t)agent * K * N * NW;
    const int Ta = T[agent];
    const DiagDesc dsc = desc[(size_t)agent * D + d];
    for (int it = threadIdx.x; it < dsc.n * K; it += blockDim.x) {
        const int g = it / K, k = it - g * K;
        float s = 0.f;
        for (int t = 0; t < Ta; ++t) {
            const float2 c = __ldg(C + dsc.coff + ((size_t)t * dsc.n_pad + g) * K + k);
            s = fmaf(c.x, c.x, fmaf(c.y, c.y, s));
        }
        const int sl = slot[dsc.slot_off + g];
        const int f = sl & 0xff, sc = (sl >> 8) & 0xff;
        W[((size_t)k * N + f) * NW + sc] = s;
        W[((size_t)k * N + sc) * NW + f] = s;
    }
}

// Sufficient statistics per (agent, diagonal), one pass over its visibilities and coherencies:
// U_k[e] = sum_t conj(c_tk) V_t[e] and the packed S_kl = sum_t conj(c_tk) c_tl (l >= k). Thread
// (slot g, direction k) accumulates U_k (4 entries) and row k of S over the samples (the threads of
// one slot share the loads of V_t and of the slot's K coherencies). STAGED: the CTA's whole V and C
// block (contiguous, [T_a][n_pad][4] and [T_a][n_pad][K]) arrives in shared memory by two bulk
// copies on one mbarrier, so every CTA has its bytes in flight at once; otherwise the samples are
// read from global memory, two in flight per thread. Written into the full circulant layout:
// compacted slot g goes to position i = its first station. Positions of flagged baselines are
// never written (they hold the zeros set when the layout was built). KB >= K: register bucket.
// Largest V + C block staged whole in shared memory; even one CTA per SM keeps far more bytes in
// flight than the streaming loop.
constexpr size_t SS_STATS_STAGED_MAX = 200 * 1024;

template <int KB, bool STAGED>
__global__ void __launch_bounds__(512, KB > 8 ? 1 : 2) k_ss_stats(const float2* __restrict__ V, const float2* __restrict__ C,
                                                                   float2* __restrict__ U, float2* __restrict__ S,
                                                                   const DiagDesc* desc, const int* slot, const int* T,
                                                                   int D, int K, int NP, int* status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    const int d = blockIdx.x, agent = blockIdx.y;
    const DiagDesc dsc = desc[(size_t)agent * D + d];
    if (dsc.n == 0) return;
    const int Ta = T[agent];
    const int KK = K * (K + 1) / 2;
    const size_t blk = ((size_t)agent * D + d) * NP;  // first position of this (agent, diagonal)
    const uint32_t vbytes = (uint32_t)Ta * dsc.n_pad * 32, cbytes = (uint32_t)Ta * dsc.n_pad * K * 8;
    const float4* Vb = reinterpret_cast<const float4*>(V + dsc.voff);
    const float2* Cb = C + dsc.coff;
    if (STAGED) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
            mbar_expect_tx(&bar, vbytes + cbytes);
            bulk_g2s(smem, Vb, vbytes, &bar);
            bulk_g2s(smem + vbytes, Cb, cbytes, &bar);
        }
        __syncthreads();
        const bool ok = mbar_wait_bounded(&bar, 0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(status, STATUS_TIMEOUT);
                mbar_wait_bounded(&bar, 0);  // the copies in flight still target this CTA's memory
            }
            return;
        }
        Vb = reinterpret_cast<const float4*>(smem);
        Cb = reinterpret_cast<const float2*>(smem + vbytes);
    }
    auto ld4 = [](const float4* p) { return STAGED ? *p : __ldg(p); };
    auto ld2 = [](const float2* p) { return STAGED ? *p : __ldg(p); };
    for (int it = threadIdx.x; it < dsc.n * K; it += blockDim.x) {
        const int g = it / K, k = it - g * K;
        float2 u[4], srow[KB];
#pragma unroll
        for (int e = 0; e < 4; ++e) u[e] = make_float2(0.f, 0.f);
#pragma unroll
        for (int l = 0; l < KB; ++l) srow[l] = make_float2(0.f, 0.f);
        const float4* vp = Vb + (size_t)g * 2;
        const float2* cp = Cb + (size_t)g * K;
        const size_t vstride = (size_t)dsc.n_pad * 2, cstride = (size_t)dsc.n_pad * K;
        auto accumulate = [&](float4 v0, float4 v1, const float2* c) {
            const float2 ck = ld2(c + k);
            const float2 vv[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                                  make_float2(v1.z, v1.w)};
#pragma unroll
            for (int e = 0; e < 4; ++e) {  // conj(c_k) V
                u[e].x = fmaf(ck.x, vv[e].x, fmaf(ck.y, vv[e].y, u[e].x));
                u[e].y = fmaf(ck.x, vv[e].y, fmaf(-ck.y, vv[e].x, u[e].y));
            }
#pragma unroll
            for (int l = 0; l < KB; ++l) {  // conj(c_k) c_l, l >= k
                if (l < k || l >= K) continue;
                const float2 cl = ld2(c + l);
                srow[l].x = fmaf(ck.x, cl.x, fmaf(ck.y, cl.y, srow[l].x));
                srow[l].y = fmaf(ck.x, cl.y, fmaf(-ck.y, cl.x, srow[l].y));
            }
        };
        int t = 0;
        for (; t + 1 < Ta; t += 2) {
            const float4 a0 = ld4(vp + t * vstride), a1 = ld4(vp + t * vstride + 1);
            const float4 b0 = ld4(vp + (t + 1) * vstride), b1 = ld4(vp + (t + 1) * vstride + 1);
            accumulate(a0, a1, cp + t * cstride);
            accumulate(b0, b1, cp + (t + 1) * cstride);
        }
        if (t < Ta) accumulate(ld4(vp + t * vstride), ld4(vp + t * vstride + 1), cp + t * cstride);
        const size_t pos = blk + (slot[dsc.slot_off + g] & 0xff);
        float4* uo = reinterpret_cast<float4*>(U + (pos * K + k) * 4);
        uo[0] = make_float4(u[0].x, u[0].y, u[1].x, u[1].y);
        uo[1] = make_float4(u[2].x, u[2].y, u[3].x, u[3].y);
        float2* so = S + pos * KK + (size_t)k * K - k * (k - 1) / 2;  // entry (k, l) at so[l - k]
#pragma unroll
        for (int l = 0; l < KB; ++l)
            if (l >= k && l < K) so[l - k] = srow[l];
    }
}

__global__ void k_check_finite(const float* x, long long n, int* status) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (; i < n; i += stride) bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, 2);
}

}  // namespace

cudaError_t prepare_data_kernels() {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int st = (int)SS_STATS_STAGED_MAX;
    cudaError_t e = cudaFuncSetAttribute(k_predict, attr, 100 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_stats<4, true>, attr, st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_stats<8, true>, attr, st);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_stats<MAX_K, true>, attr, st);
    return e;
}

cudaError_t launch_ingest(const IngestArgs& a, cudaStream_t s) {
    dim3 grid(a.D, a.A);
    k_ingest<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_extract_coh(const IngestArgs& a, float2* user_dst, cudaStream_t s) {
    dim3 grid(a.D, a.A);
    k_extract_coh<<<grid, 256, 0, s>>>(a, user_dst);
    return cudaGetLastError();
}
cudaError_t launch_residual(const ResidualArgs& a, cudaStream_t s) {
    dim3 grid(a.D, a.A);
    k_residual<<<grid, RES_THREADS, (size_t)a.K * 2 * RES_THREADS * sizeof(float4), s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_predict(const PredictArgs& a, cudaStream_t s) {
    const size_t budget = 96 * 1024;
    int s_chunk = a.S;
    // per source: its N station phasors (8 B each), its flux (4 B) and l, m, n - 1 (24 B)
    while (s_chunk > 1 && (size_t)a.K * s_chunk * (a.N * 8 + 28) > budget) s_chunk = (s_chunk + 1) / 2;
    const size_t smem = (size_t)a.K * s_chunk * (a.N * 8 + 28);
    dim3 grid(a.Tmax, a.A);
    k_predict<<<grid, 256, smem, s>>>(a, s_chunk);
    return cudaGetLastError();
}
cudaError_t launch_gram_weights(const float2* C, const DiagDesc* desc, const int* slot, const int* T, float* gw,
                                int A, int D, int K, int N, cudaStream_t s) {
    const cudaError_t e = cudaMemsetAsync(gw, 0, (size_t)A * K * N * ((N + 3) / 4 * 4) * sizeof(float), s);
    if (e != cudaSuccess) return e;
    k_gram_weights<<<dim3(D, A), 128, 0, s>>>(C, desc, slot, T, gw, D, K, N);
    return cudaGetLastError();
}
// Shared memory of a CTA of the staged statistics pass: the largest V + C block.
size_t ss_stats_smem(int N, int K, int Tmax) { return (size_t)Tmax * ((N + 3) / 4 * 4) * (32 + 8 * K); }

template <int KB>
cudaError_t ss_stats_go(const float2* V, const float2* C, float2* U, float2* S, const DiagDesc* desc, const int* slot,
                        const int* T, int A, int D, int K, int NP, size_t smem, int* status, cudaStream_t s) {
    const int threads = std::min(512, ((NP * K + 31) / 32) * 32);
    dim3 grid(D, A);
    if (smem <= SS_STATS_STAGED_MAX)
        k_ss_stats<KB, true><<<grid, threads, smem, s>>>(V, C, U, S, desc, slot, T, D, K, NP, status);
    else
        k_ss_stats<KB, false><<<grid, threads, 0, s>>>(V, C, U, S, desc, slot, T, D, K, NP, status);
    return cudaGetLastError();
}

cudaError_t launch_ss_stats(const float2* V, const float2* C, float2* U, float2* S, const DiagDesc* desc,
                            const int* slot, const int* T, int A, int D, int K, int N, int Tmax, int* status,
                            cudaStream_t s) {
    const int NP = (N + 3) / 4 * 4;
    const size_t smem = ss_stats_smem(N, K, Tmax);
    if (K <= 4) return ss_stats_go<4>(V, C, U, S, desc, slot, T, A, D, K, NP, smem, status, s);
    if (K <= 8) return ss_stats_go<8>(V, C, U, S, desc, slot, T, A, D, K, NP, smem, status, s);
    return ss_stats_go<MAX_K>(V, C, U, S, desc, slot, T, A, D, K, NP, smem, status, s);
}

cudaError_t launch_check_finite(const float* x, long long n, int* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<(unsigned)blocks, 256, 0, s>>>(x, n, status);
    return cudaGetLastError();
}

}  // namespace calib
