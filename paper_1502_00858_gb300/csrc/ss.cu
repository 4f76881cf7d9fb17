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
//
// Work split: the A*D (agent, circulant diagonal) items are cut into gridDim.x equal contiguous
// ranges, one per CTA, and the grid is a multiple of the SM count, so every SM gets the same work
// and there is no partial last wave. The statistics are in the full circulant layout (slot i of
// diagonal d is the pair (i, (i+d) mod N), zero statistics where flagged), so thread pair g owns
// station g as the first station of its slot in every diagonal: it keeps that station's rows of
// J and eta (or the trial point J') and its first-station sums in registers for the whole agent, and only the
// second station (g+d) mod N goes through shared memory. A CTA stages J and eta of its current
// agent, streams the per-slot statistics of one diagonal per stage through a cp.async.bulk ring
// (mbarrier, bounded waits), and writes the station sums as one partial per (agent, piece) when
// the agent changes; piece = the CTA's index among the CTAs whose range meets that agent.
// Two threads per slot, one per row of the 2x2 blocks: thread rr forms row rr of Q_l (or P_l and
// dP_l), of the S-weighted sums X_k and of both station terms; the second station's term
// X_k^H J_f needs column rr of X_k, whose other entry comes from the partner lane. Within a
// diagonal every station is the second element of at most one slot, so the shared-memory updates
// of a diagonal are conflict-free (no atomics). The trial pass reads J' and forms the step as
// x = J' - J (dP_l = x_pl J'_ql^H + J_pl x_ql^H, the same model change).
#include "ss_common.cuh"

namespace calib {
namespace {

using namespace ss;

// KB: register bucket; EXACT: K == KB, so every loop bound and packed-S index is a constant.
// SMALL: at most 128 threads (N <= 64): 168 registers with 3 CTAs of 128 threads per SM (the trial
// pass's shared memory allows 3; the Hessian pass spends the registers on loads hoisted ahead of
// their use); from K = 8 on, shared memory allows 2 CTAs (K = 8) or 1 (K >= 10) and the register
// budget follows. Larger CTAs: 128 registers for the Hessian pass (2 CTAs of 256), unbounded for the trial.
// Stage layout: [U: n2][K][2 rows] float4 (trial only) | [S: n2][KK] float2, n2 = the diagonal's slot
// count rounded up to even.
template <int KB, bool HV, bool EXACT, bool SMALL>
__global__ void __launch_bounds__(SMALL ? 128 : 256,
                                  SMALL ? (KB >= 10 ? (ss_u_global(HV, KB) ? 2 : 1) : (KB >= 8 ? 2 : 3)) : (HV ? 2 : 1))
    k_ss_sweep(const SSArgs a, const int stage_bytes) {
    constexpr int NST = nst<HV>();
    constexpr float sg = HV ? 1.f : -1.f;  // station terms: + in the Hessian pass, - (gradient) in the trial pass
    constexpr bool UG = ss_u_global(HV, KB);  // the trial pass reads U from global memory (not staged)
    extern __shared__ __align__(128) unsigned char smem[];
    const int N = a.N, D = a.D, NP = a.NP;
    const int K = EXACT ? KB : a.K;
    const int KK = K * (K + 1) / 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int g = tid >> 1, rr = tid & 1, ro = rr ^ 1;
    const int lane = tid & 31;
    const int KN2 = K * N * 2;  // float4 per vector: [K][N][row]
    const bool own = g < N;     // this thread pair owns station g

    unsigned char* stage = smem;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + NST * stage_bytes);
    float4* Js = reinterpret_cast<float4*>(smem + NST * stage_bytes + BAR_BYTES);  // [K][N][2 rows]
    float4* Es = Js + KN2;     // eta (Hessian) or the trial point J' = J + x (trial)
    float4* accs = Es + KN2;   // second-station sums
    double* red = reinterpret_cast<double*>(accs + KN2);  // [32]

    const long long W = (long long)a.A * D, G = gridDim.x;
    const long long i0 = (long long)blockIdx.x * W / G;
    const int S = (int)((long long)(blockIdx.x + 1) * W / G - i0);
    const int ag0 = (int)(i0 / D), d0 = (int)(i0 - (long long)ag0 * D);  // d0: 0-based diagonal

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) mbar_init(&bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Thread 0 issues the stages in order; (iss_ag, iss_d) is the item of the next one.
    int iss_ag = ag0, iss_d = d0;
    const uint64_t pol = tid == 0 ? l2_evict_first() : 0ull;
    auto issue = [&](int s2) {
        const size_t blk = ((size_t)iss_ag * D + iss_d) * NP;
        const int n = (2 * (iss_d + 1) == N) ? N / 2 : N;
        const int n2 = (n + 1) & ~1;  // an even slot count keeps both copies multiples of 16 bytes
        if (++iss_d == D) { iss_d = 0; ++iss_ag; }
        const uint32_t ub = (HV || UG) ? 0u : (uint32_t)(n2 * K * 32);
        const uint32_t sb = (uint32_t)(n2 * KK * 8);
        unsigned char* buf = stage + (s2 % NST) * stage_bytes;
        uint64_t* b = &bar[s2 % NST];
        mbar_expect_tx(b, ub + sb);
        if (!HV) bulk_g2s_stream(buf, a.U + blk * K * 4, ub, b, pol);
        bulk_g2s_stream(buf + ub, a.S + blk * KK, sb, b, pol);
    };
    if (tid == 0)
        for (int s2 = 0; s2 < min(NST - 1, S); ++s2) issue(s2);
    // Everything above reads only the statistics; J, eta (or J') and the partial buffers belong to
    // the preceding kernels of the chain (programmatic dependent launch).
    griddep_wait();
    griddep_launch_dependents();

    float4 Jf[KB], Ef[KB], A1[KB];  // rows rr of station g's J and eta / J'; its first-station sums
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < KB; ++k) Jf[k] = Ef[k] = A1[k] = z4;

    // Station sums of the finished agent -> its partial; call from uniform control flow after a barrier.
    auto flush = [&](int ag, double dc) {
        const long long piece = blockIdx.x - cta_of_item((long long)ag * D, W, G);
        const size_t slot_p = (size_t)ag * a.part_stride + (size_t)piece;
        float4* out = reinterpret_cast<float4*>(a.part) + slot_p * KN2;
        if (own) {
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
                const int i = (k * N + g) * 2 + rr;
                const float4 w = accs[i];
                out[i] = make_float4(A1[k].x + w.x, A1[k].y + w.y, A1[k].z + w.z, A1[k].w + w.w);
            }
        }
        if (!HV) {
            for (int o = 16; o > 0; o >>= 1) dc += __shfl_down_sync(0xffffffffu, dc, o);
            if (lane == 0) red[tid >> 5] = dc;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < (nthr >> 5); ++w) t += red[w];
                a.part_dcost[slot_p] = t;
            }
        }
    };

    int agent = -1, ag = ag0, dg = d0;  // current agent with staged J / eta; item of stage s
    bool fresh = false;
    double dcost = 0.0;
    for (int s = 0; s < S; ++s) {
        if (ag != agent) {
            if (agent >= 0) {
                __syncthreads();  // every thread is done with the previous agent's sums
                flush(agent, dcost);
                dcost = 0.0;
                __syncthreads();  // the sums are read out before they are cleared
            }
            agent = ag;
            fresh = true;
            const float4* Jg = reinterpret_cast<const float4*>(a.J) + (size_t)ag * KN2;
            const float4* Eg = reinterpret_cast<const float4*>(a.eta) + (size_t)ag * KN2;
            for (int i = tid; i < KN2; i += nthr) {
                Js[i] = __ldg(Jg + i);
                Es[i] = __ldg(Eg + i);
                accs[i] = z4;
            }
        }
        const int d = dg + 1;  // circulant diagonal of this stage
        if (++dg == D) { dg = 0; ++ag; }
        const bool ok = mbar_wait_bounded(&bar[s % NST], (uint32_t)((s / NST) & 1));
        // One barrier per stage: stage s has landed everywhere, every thread is done with stage
        // s - 1 (its buffer is free for stage s + 1), and the agent's J / eta are staged.
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
        if (fresh) {  // station g's rows of the new agent
            fresh = false;
            if (own) {
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k >= K) continue;
                    Jf[k] = Js[(k * N + g) * 2 + rr];
                    Ef[k] = Es[(k * N + g) * 2 + rr];
                    A1[k] = z4;
                }
            }
        }
        const int n = (2 * d == N) ? N / 2 : N;
        const int n2 = (n + 1) & ~1;
        const unsigned char* buf = stage + (s % NST) * stage_bytes;
        // U of this diagonal [n2][K][2][2] (trial): staged, or read from global memory (UG)
        const float2* Us = UG ? a.U + ((size_t)agent * D + (d - 1)) * NP * K * 4 : reinterpret_cast<const float2*>(buf);
        const float2* Ss = reinterpret_cast<const float2*>(buf + ((HV || UG) ? 0 : n2 * K * 32)) + (size_t)g * KK;
        const bool active = g < n;
        const int second = (g + d < N) ? g + d : g + d - N;
        // Row rr of X_k in column order (rr, 1 - rr): Hessian (S Q)_k; trial W'_k = U_k - (S P)_k - (S dP)_k.
        float2 Xd[KB], Xo[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) Xd[k] = Xo[k] = make_float2(0.f, 0.f);
        if (active) {
            float2 Yd[HV ? 1 : KB], Yo[HV ? 1 : KB];    // trial: row rr of (S dP)_k
            float2 dPd[HV ? 1 : KB], dPo[HV ? 1 : KB];  // trial: row rr of dP_l
            if (!HV) {
#pragma unroll
                for (int k = 0; k < KB; ++k) Yd[k] = Yo[k] = dPd[k] = dPo[k] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int l = 0; l < KB; ++l) {
                if (l >= K) continue;
                // rows rr and 1 - rr of the second station's blocks; (A B^H)[rr][c] = A[rr][0] conj(B[c][0]) +
                // A[rr][1] conj(B[c][1]) for the columns c = rr (d) and 1 - rr (o)
                const float4 jsd = Js[(l * N + second) * 2 + rr], jso = Js[(l * N + second) * 2 + ro];
                const float4 esd = Es[(l * N + second) * 2 + rr], eso = Es[(l * N + second) * 2 + ro];
                const float2 z2 = make_float2(0.f, 0.f);
                float2 qd, qo, pd = z2, po = z2;
                if (HV) {  // Q_l = eta_f J_s^H + J_f eta_s^H
                    qd = cdot2_acc(cdot2_acc(z2, Ef[l], jsd), Jf[l], esd);
                    qo = cdot2_acc(cdot2_acc(z2, Ef[l], jso), Jf[l], eso);
                } else {   // P_l = J_f J_s^H;  dP_l = J'_f J'_s^H - P_l = x_f J'_s^H + J_f x_s^H, x = J' - J
                    const float4 xf = f4sub(Ef[l], Jf[l]);
                    qd = cdot2_acc(z2, Jf[l], jsd);
                    qo = cdot2_acc(z2, Jf[l], jso);
                    pd = cdot2_acc(cdot2_acc(z2, xf, esd), Jf[l], f4sub(esd, jsd));
                    po = cdot2_acc(cdot2_acc(z2, xf, eso), Jf[l], f4sub(eso, jso));
                    dPd[l] = pd;
                    dPo[l] = po;
                }
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k >= K) continue;
                    // S_kl from the packed upper triangle; S_kl = conj(S_lk) below the diagonal
                    const int lo = k < l ? k : l, hi = k < l ? l : k;
                    float2 skl = Ss[lo * K - lo * (lo - 1) / 2 + (hi - lo)];
                    if (k > l) skl.y = -skl.y;
                    cmac(Xd[k], skl, qd);
                    cmac(Xo[k], skl, qo);
                    if (!HV) {
                        cmac(Yd[k], skl, pd);
                        cmac(Yo[k], skl, po);
                    }
                }
            }
            if (!HV) {
                float dcf = 0.f;
#pragma unroll
                for (int k = 0; k < KB; ++k) {
                    if (k >= K) continue;
                    const float2* u = Us + (((size_t)g * K + k) * 2 + rr) * 2;
                    const float2 ud = UG ? __ldg(u + rr) : u[rr], uo = UG ? __ldg(u + ro) : u[ro];
                    const float2 Wd = f2sub(ud, Xd[k]);  // W_k at J
                    const float2 Wo = f2sub(uo, Xo[k]);
                    // decrease: Re[conj(dP_k) (2 W_k - (S dP)_k)], this row
                    dcf = fmaf(dPd[k].x, 2.f * Wd.x - Yd[k].x, fmaf(dPd[k].y, 2.f * Wd.y - Yd[k].y, dcf));
                    dcf = fmaf(dPo[k].x, 2.f * Wo.x - Yo[k].x, fmaf(dPo[k].y, 2.f * Wo.y - Yo[k].y, dcf));
                    Xd[k] = f2sub(Wd, Yd[k]);  // W'_k at J' = J + x
                    Xo[k] = f2sub(Wo, Yo[k]);
                }
                dcost += (double)dcf;
            }
        }
        // Station terms, row rr (J' = J + x in the trial pass; Hessian: +, trial: -):
        //   first (g, registers): (X J'_s)[rr][.] = X[rr][rr] J'_s[rr][.] + X[rr][1-rr] J'_s[1-rr][.]
        //   second (shared):      (X^H J'_f)[rr][.] = conj(X[rr][rr]) J'_f[rr][.] + conj(X[1-rr][rr]) J'_f[1-rr][.]
        // X[1-rr][rr] is the partner lane's Xo; J'_f[rr] is in registers, J'_f[1-rr] in shared memory.
        const float4* Jp = HV ? Js : Es;  // J' (the Hessian pass is taken at J)
        if constexpr (KB <= 5) {
            // Every second-station sum is read before any is written: the compiler cannot tell the
            // directions' addresses apart and would otherwise wait for each store before the next
            // load. (Larger buckets have no registers to spare for this.)
            float2 xp[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k) xp[k] = k < K ? shfl2x(Xo[k]) : make_float2(0.f, 0.f);
            if (!active) continue;
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
                const float4 sd = Jp[(k * N + second) * 2 + rr], so = Jp[(k * N + second) * 2 + ro];
                const float2 a0 = cmul2_acc(make_float2(A1[k].x, A1[k].y), sg, Xd[k], make_float2(sd.x, sd.y), Xo[k], make_float2(so.x, so.y));
                const float2 a1 = cmul2_acc(make_float2(A1[k].z, A1[k].w), sg, Xd[k], make_float2(sd.z, sd.w), Xo[k], make_float2(so.z, so.w));
                A1[k] = make_float4(a0.x, a0.y, a1.x, a1.y);
            }
            float4 t2[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k) t2[k] = k < K ? accs[(k * N + second) * 2 + rr] : z4;
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
                const float4 fd = HV ? Jf[k] : Ef[k], fo = Jp[(k * N + g) * 2 + ro];
                const float2 b0 = cmul2c_acc(make_float2(t2[k].x, t2[k].y), sg, Xd[k], make_float2(fd.x, fd.y), xp[k], make_float2(fo.x, fo.y));
                const float2 b1 = cmul2c_acc(make_float2(t2[k].z, t2[k].w), sg, Xd[k], make_float2(fd.z, fd.w), xp[k], make_float2(fo.z, fo.w));
                accs[(k * N + second) * 2 + rr] = make_float4(b0.x, b0.y, b1.x, b1.y);
            }
        } else {
#pragma unroll
            for (int k = 0; k < KB; ++k) {
                if (k >= K) continue;
                const float2 xp = shfl2x(Xo[k]);
                if (!active) continue;
                const float4 sd = Jp[(k * N + second) * 2 + rr], so = Jp[(k * N + second) * 2 + ro];
                const float4 fd = HV ? Jf[k] : Ef[k], fo = Jp[(k * N + g) * 2 + ro];
                const float2 a0 = cmul2_acc(make_float2(A1[k].x, A1[k].y), sg, Xd[k], make_float2(sd.x, sd.y), Xo[k], make_float2(so.x, so.y));
                const float2 a1 = cmul2_acc(make_float2(A1[k].z, A1[k].w), sg, Xd[k], make_float2(sd.z, sd.w), Xo[k], make_float2(so.z, so.w));
                A1[k] = make_float4(a0.x, a0.y, a1.x, a1.y);
                float4* d2 = accs + (k * N + second) * 2 + rr;
                const float4 t2 = *d2;
                const float2 b0 = cmul2c_acc(make_float2(t2.x, t2.y), sg, Xd[k], make_float2(fd.x, fd.y), xp, make_float2(fo.x, fo.y));
                const float2 b1 = cmul2c_acc(make_float2(t2.z, t2.w), sg, Xd[k], make_float2(fd.z, fd.w), xp, make_float2(fo.z, fo.w));
                *d2 = make_float4(b0.x, b0.y, b1.x, b1.y);
            }
        }
    }
    if (agent >= 0) {
        __syncthreads();
        flush(agent, dcost);
    }
}

template <int KB, bool HV>
cudaError_t prep_kb() {
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_ss_sweep<KB, HV, true, false>, attr, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_sweep<KB, HV, false, false>, attr, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_sweep<KB, HV, true, true>, attr, 200 * 1024);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ss_sweep<KB, HV, false, true>, attr, 200 * 1024);
    return e;
}
template <bool HV>
cudaError_t prep_all() {
    cudaError_t e;
    if constexpr (!HV) {  // the Hessian pass for K <= HV1_KMAX runs k_ss_hessvec
        if ((e = prep_kb<1, HV>()) != cudaSuccess) return e;
        if ((e = prep_kb<2, HV>()) != cudaSuccess) return e;
        if ((e = prep_kb<3, HV>()) != cudaSuccess) return e;
        if ((e = prep_kb<4, HV>()) != cudaSuccess) return e;
        if ((e = prep_kb<5, HV>()) != cudaSuccess) return e;
    }
    if ((e = prep_kb<6, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<8, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<10, HV>()) != cudaSuccess) return e;
    if ((e = prep_kb<12, HV>()) != cudaSuccess) return e;
    return prep_kb<16, HV>();
}

template <int KB, bool HV>
cudaError_t go(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s) {
    const bool exact = a.K == KB, small = threads <= 128, pdl = a.pdl != 0;
    if (exact && small) return launch_k(pdl, k_ss_sweep<KB, HV, true, true>, grid, threads, smem, s, a, sb);
    if (exact) return launch_k(pdl, k_ss_sweep<KB, HV, true, false>, grid, threads, smem, s, a, sb);
    if (small) return launch_k(pdl, k_ss_sweep<KB, HV, false, true>, grid, threads, smem, s, a, sb);
    return launch_k(pdl, k_ss_sweep<KB, HV, false, false>, grid, threads, smem, s, a, sb);
}
template <bool HV>
cudaError_t dispatch(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s) {
    const int K = a.K;
    if constexpr (!HV) {
        if (K <= 1) return go<1, HV>(a, grid, threads, smem, sb, s);
        if (K <= 2) return go<2, HV>(a, grid, threads, smem, sb, s);
        if (K <= 3) return go<3, HV>(a, grid, threads, smem, sb, s);
        if (K <= 4) return go<4, HV>(a, grid, threads, smem, sb, s);
        if (K <= 5) return go<5, HV>(a, grid, threads, smem, sb, s);
    }
    if (K <= 6) return go<6, HV>(a, grid, threads, smem, sb, s);
    if (K <= 8) return go<8, HV>(a, grid, threads, smem, sb, s);
    if (K <= 10) return go<10, HV>(a, grid, threads, smem, sb, s);
    if (K <= 12) return go<12, HV>(a, grid, threads, smem, sb, s);
    return go<16, HV>(a, grid, threads, smem, sb, s);
}

}  // namespace

cudaError_t prepare_ss_kernels() {
    cudaError_t e = prep_all<false>();
    if (e == cudaSuccess) e = prep_all<true>();
    if (e == cudaSuccess) e = prepare_ss_hessvec_kernels();
    return e;
}

size_t ss_sweep_smem_bytes(int N, int K, bool hessvec, int* stage_bytes) {
    const int KK = K * (K + 1) / 2, N2 = (N + 1) / 2 * 2;  // slots copied per stage (even)
    const int per_slot = ((hessvec || ss_u_global(false, ss_bucket(K))) ? 0 : K * 32) + KK * 8;
    const int sb = ((N2 * per_slot + 127) / 128) * 128;
    if (stage_bytes) *stage_bytes = sb;
    const int nstages = hessvec ? nst<true>() : nst<false>();
    // the one-thread-per-slot Hessian kernel needs no reduction area
    const int red = (hessvec && K <= HV1_KMAX) ? 0 : 32 * 8;
    return (size_t)nstages * sb + BAR_BYTES + (size_t)3 * K * N * 32 + red;
}

int ss_sweep_threads(int N) { return ((2 * ((N + 3) / 4 * 4) + 31) / 32) * 32; }

cudaError_t launch_ss_sweep(const SSArgs& a, bool hessvec, int grid, cudaStream_t s) {
    int sb = 0;
    const size_t smem = ss_sweep_smem_bytes(a.N, a.K, hessvec, &sb);
    if (smem > 200 * 1024 || grid < 1 || (long long)grid > (long long)a.A * a.D) return cudaErrorInvalidConfiguration;
    if (hessvec && a.K <= HV1_KMAX) return launch_ss_hessvec1(a, grid, (a.N + 31) / 32 * 32, smem, sb, s);
    const int threads = ss_sweep_threads(a.N);
    return hessvec ? dispatch<true>(a, grid, threads, smem, sb, s) : dispatch<false>(a, grid, threads, smem, sb, s);
}

}  // namespace calib
