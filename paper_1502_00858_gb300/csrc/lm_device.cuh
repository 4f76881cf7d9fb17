// Device-side pieces of the per-agent Levenberg-Marquardt / PCG logic (Section 3, Eq. M1), shared by
// the stand-alone kernels (lm.cu) and the sweeps that finish an agent's LM/PCG step in the last CTA to
// complete its chunks (ss.cu). See lm.cu for the method. Every function uses all threads of the CTA
// (blockDim a multiple of 32) and contains block barriers: call it from uniform control flow.
#pragma once

#include <math.h>

#include "calib_internal.cuh"

namespace calib {
namespace {


__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

__device__ double block_max(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = red[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s = fmax(s, red[i]);
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

struct Blk { float v[8]; };

__device__ __forceinline__ Blk load_blk(const float* base, int blk) {
    Blk b;
    const float4* p = reinterpret_cast<const float4*>(base + (size_t)blk * 8);
    const float4 a0 = p[0], a1 = p[1];
    b.v[0] = a0.x; b.v[1] = a0.y; b.v[2] = a0.z; b.v[3] = a0.w;
    b.v[4] = a1.x; b.v[5] = a1.y; b.v[6] = a1.z; b.v[7] = a1.w;
    return b;
}
__device__ __forceinline__ void store_blk(float* base, int blk, const Blk& b) {
    float4* p = reinterpret_cast<float4*>(base + (size_t)blk * 8);
    p[0] = make_float4(b.v[0], b.v[1], b.v[2], b.v[3]);
    p[1] = make_float4(b.v[4], b.v[5], b.v[6], b.v[7]);
}
// Per-block dot products are float32 (8 terms); each thread sums its blocks in float32 and the
// cross-thread reduction is float64 (float64 arithmetic is scarce on this GPU).
__device__ __forceinline__ float dot_blk(const Blk& a, const Blk& b) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s = fmaf(a.v[i], b.v[i], s);
    return s;
}

// x (G + lam I)^-1 for a 2x2 complex block x (row-major re,im pairs) and Hermitian G (g00, g11, re g01, im g01).
__device__ __forceinline__ Blk precond(const Blk& x, const float* G, float lam) {
    const float a = G[0] + lam, c = G[1] + lam, br = G[2], bi = G[3];
    const float id = 1.f / (a * c - (br * br + bi * bi));
    // Minv = id * [[c, -b], [-conj(b), a]]  (m00, m11 real)
    const float m00 = c * id, m01r = -br * id, m01i = -bi * id;
    const float m10r = -br * id, m10i = bi * id, m11 = a * id;
    Blk z;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const float x0r = x.v[r * 4 + 0], x0i = x.v[r * 4 + 1], x1r = x.v[r * 4 + 2], x1i = x.v[r * 4 + 3];
        // z[r][0] = x[r][0] m00 + x[r][1] m10 ; z[r][1] = x[r][0] m01 + x[r][1] m11
        z.v[r * 4 + 0] = x0r * m00 + x1r * m10r - x1i * m10i;
        z.v[r * 4 + 1] = x0i * m00 + x1r * m10i + x1i * m10r;
        z.v[r * 4 + 2] = x0r * m01r - x0i * m01i + x1r * m11;
        z.v[r * 4 + 3] = x0r * m01i + x0i * m01r + x1i * m11;
    }
    return z;
}

// Sum of the per-chunk partial station sums of a sweep, fixed chunk order.
__device__ __forceinline__ Blk sum_parts(const LMArgs& a, int agent, int blk, int KN) {
    Blk s;
#pragma unroll
    for (int i = 0; i < 8; ++i) s.v[i] = 0.f;
    for (int ch = 0; ch < a.n_chunks; ++ch) {
        // L2-coherent loads: in a fused sweep other CTAs wrote these partials during this launch
        const float4* q = reinterpret_cast<const float4*>(a.part + ((size_t)agent * a.n_chunks + ch) * KN * 8) + 2 * blk;
        const float4 q0 = __ldcg(q), q1 = __ldcg(q + 1);
        const Blk p = {{q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w}};
#pragma unroll
        for (int i = 0; i < 8; ++i) s.v[i] += p.v[i];
    }
    return s;
}

// Penalty Re tr(Y^H D) + rho/2 ||D||^2, D = J - BZ (Eq. sumtrace2), this thread's share.
__device__ double penalty_part(const float* J, const float* Y, const float* BZ, const float* rho,
                               int N, int KN) {
    float pen = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const int k = blk / N;
        const Blk j = load_blk(J, blk), y = load_blk(Y, blk), bz = load_blk(BZ, blk);
        float yd = 0.f, dd = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float d = j.v[i] - bz.v[i];
            yd = fmaf(y.v[i], d, yd);
            dd = fmaf(d, d, dd);
        }
        pen += yd + 0.5f * rho[k] * dd;
    }
    return (double)pen;
}

// Decrease of the penalty from J to Jt, pen(J) - pen(Jt) = -(Re tr(Y^H x) + rho Re tr(D^H x) + rho/2 ||x||^2)
// with D = J - BZ and x = Jt - J, this thread's share. Formed from the small x, so it is accurate
// relative to the decrease itself.
__device__ double penalty_decrease_part(const float* J, const float* Jt, const float* Y, const float* BZ,
                                        const float* rho, int N, int KN) {
    float s = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const float rk = rho[blk / N];
        const Blk j = load_blk(J, blk), jt = load_blk(Jt, blk), y = load_blk(Y, blk), bz = load_blk(BZ, blk);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float x = jt.v[i] - j.v[i];  // exact: Jt = J + x was rounded once
            const float d = j.v[i] - bz.v[i];
            s -= fmaf(y.v[i], x, rk * fmaf(0.5f * x, x, d * x));
        }
    }
    return (double)s;
}

// Remove the component of a data gradient G_k along the gauge orbit {J_k A : A anti-Hermitian}.
// g is invariant under J_k -> J_k U (C = c I_2, Eq. coh), so its exact gradient has none: the
// anti-Hermitian part of J_k^H G_k vanishes. Float32 residuals leave round-off there, which would
// otherwise steer the weakly determined gauge mode (curved only by the rho/2 penalty). With
// S = J^H J, solve (S A + A S)/2 = skew(J^H G) for A = [[i a, b + i c], [-b + i c, i d]] and set
// G <- G - J A (the h-orthogonal projection). Exact arithmetic leaves G unchanged.
// One warp per direction (warp-level float64 reductions, no block barriers until the end).
__device__ void project_out_gauge(const float* J, float* G, int N, int K) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = warp; k < K; k += nwarps) {
        const float* Jk = J + (size_t)k * N * 8;
        float* Gk = G + (size_t)k * N * 8;
        double v[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = 0.0;
        for (int p = lane; p < N; p += 32) {
            const float* j = Jk + p * 8;
            const float* g = Gk + p * 8;
            // S += J^H J (s0, s1, re s01, im s01); M += J^H G (4 complex, row-major)
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const double j0r = j[m * 4 + 0], j0i = j[m * 4 + 1], j1r = j[m * 4 + 2], j1i = j[m * 4 + 3];
                v[0] += j0r * j0r + j0i * j0i;
                v[1] += j1r * j1r + j1i * j1i;
                v[2] += j0r * j1r + j0i * j1i;
                v[3] += j0r * j1i - j0i * j1r;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const double gr = g[m * 4 + 2 * c], gi = g[m * 4 + 2 * c + 1];
                    v[4 + 2 * c] += j0r * gr + j0i * gi;  // M[0][c] += conj(J[m][0]) G[m][c]
                    v[5 + 2 * c] += j0r * gi - j0i * gr;
                    v[8 + 2 * c] += j1r * gr + j1i * gi;  // M[1][c] += conj(J[m][1]) G[m][c]
                    v[9 + 2 * c] += j1r * gi - j1i * gr;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 12; ++i)
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        double sol[4] = {0.0, 0.0, 0.0, 0.0};
        if (lane == 0) {
            const double s0 = v[0], s1 = v[1], u = v[2], w = v[3];
            // skew(M): t0 = Im M00, t1 = Im M11, t2 + i t3 = (M01 - conj(M10)) / 2
            const double t0 = v[5], t1 = v[11];
            const double t2 = 0.5 * (v[6] - v[8]), t3 = 0.5 * (v[7] + v[9]);
            // unknowns (a, d, b, c):  a s0 + u c - w b = t0;  d s1 + u c - w b = t1;
            // (b (s0+s1) - w (a+d)) / 2 = t2;  (c (s0+s1) + u (a+d)) / 2 = t3
            double Mx[4][5] = {{s0, 0.0, -w, u, t0},
                               {0.0, s1, -w, u, t1},
                               {-0.5 * w, -0.5 * w, 0.5 * (s0 + s1), 0.0, t2},
                               {0.5 * u, 0.5 * u, 0.0, 0.5 * (s0 + s1), t3}};
            bool ok = true;
            for (int col = 0; col < 4 && ok; ++col) {
                int piv = col;
                for (int r = col + 1; r < 4; ++r)
                    if (fabs(Mx[r][col]) > fabs(Mx[piv][col])) piv = r;
                if (!(fabs(Mx[piv][col]) > 1e-30)) { ok = false; break; }
                for (int cc = 0; cc < 5; ++cc) { const double tmp = Mx[col][cc]; Mx[col][cc] = Mx[piv][cc]; Mx[piv][cc] = tmp; }
                for (int r = 0; r < 4; ++r) {
                    if (r == col) continue;
                    const double f = Mx[r][col] / Mx[col][col];
                    for (int cc = col; cc < 5; ++cc) Mx[r][cc] -= f * Mx[col][cc];
                }
            }
            if (ok)
                for (int i = 0; i < 4; ++i) sol[i] = Mx[i][4] / Mx[i][i];
        }
        const float a = (float)__shfl_sync(0xffffffffu, sol[0], 0), d = (float)__shfl_sync(0xffffffffu, sol[1], 0);
        const float b = (float)__shfl_sync(0xffffffffu, sol[2], 0), c = (float)__shfl_sync(0xffffffffu, sol[3], 0);
        // A = [[i a, b + i c], [-b + i c, i d]]
        const float A00r = 0.f, A00i = a, A01r = b, A01i = c, A10r = -b, A10i = c, A11r = 0.f, A11i = d;
        for (int p = lane; p < N; p += 32) {
            const float* j = Jk + p * 8;
            float* g = Gk + p * 8;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const float jr0 = j[r * 4 + 0], ji0 = j[r * 4 + 1], jr1 = j[r * 4 + 2], ji1 = j[r * 4 + 3];
                // (J A)[r][0] = J[r][0] A00 + J[r][1] A10 ; (J A)[r][1] = J[r][0] A01 + J[r][1] A11
                g[r * 4 + 0] -= jr0 * A00r - ji0 * A00i + jr1 * A10r - ji1 * A10i;
                g[r * 4 + 1] -= jr0 * A00i + ji0 * A00r + jr1 * A10i + ji1 * A10r;
                g[r * 4 + 2] -= jr0 * A01r - ji0 * A01i + jr1 * A11r - ji1 * A11i;
                g[r * 4 + 3] -= jr0 * A01i + ji0 * A01r + jr1 * A11i + ji1 * A11r;
            }
        }
    }
    __syncthreads();
}

// Jacobi blocks G_pk = sum over the baselines incident on p of s_bk J_ok^H J_ok (o the other station,
// s_bk = sum_t |c_btk|^2) at the current J. Each (direction, station) thread gathers over the agent's
// station-incidence list in a fixed order: no atomics and no barriers inside the sum.
__device__ void gram_blocks(const LMArgs& a, int agent, const float* J, float* Gout, float* Xs, float* Gs) {
    const int N = a.N, K = a.K, KN = K * N;
    (void)Gs;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const Blk j = load_blk(J, blk);
        // X = J^H J: x00 = |J00|^2 + |J10|^2, x11 = |J01|^2 + |J11|^2, x01 = conj(J00) J01 + conj(J10) J11
        const float j00r = j.v[0], j00i = j.v[1], j01r = j.v[2], j01i = j.v[3];
        const float j10r = j.v[4], j10i = j.v[5], j11r = j.v[6], j11i = j.v[7];
        Xs[blk * 4 + 0] = j00r * j00r + j00i * j00i + j10r * j10r + j10i * j10i;
        Xs[blk * 4 + 1] = j01r * j01r + j01i * j01i + j11r * j11r + j11i * j11i;
        Xs[blk * 4 + 2] = j00r * j01r + j00i * j01i + j10r * j11r + j10i * j11i;
        Xs[blk * 4 + 3] = j00r * j01i - j00i * j01r + j10r * j11i - j10i * j11r;
    }
    __syncthreads();
    const int* off = a.inc_off + (size_t)agent * (N + 1);
    for (int it = threadIdx.x; it < KN; it += blockDim.x) {
        const int k = it / N, p = it - k * N;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
        const int e = off[p + 1];
#pragma unroll 4
        for (int j = off[p]; j < e; ++j) {
            const int2 so = a.inc[j];  // (global slot, other station)
            const float w = a.spow[(size_t)so.x * K + k];
            const float* X = Xs + (k * N + so.y) * 4;
            g0 = fmaf(w, X[0], g0);
            g1 = fmaf(w, X[1], g1);
            g2 = fmaf(w, X[2], g2);
            g3 = fmaf(w, X[3], g3);
        }
        float* G = Gout + (size_t)it * 4;
        G[0] = g0; G[1] = g1; G[2] = g2; G[3] = g3;
    }
    __syncthreads();
}

// grad = gradg + Y/2 + rho/2 (J - BZ); r = -grad; z = M^-1 r; p = z; x = 0; rz = h(r, z).
__device__ void cg_init(const LMArgs& a, int agent, const float* G, double* red) {
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    const float mu = (float)st.mu;
    float rz = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const int k = blk / N;
        const float rk = a.rho[k];
        const Blk gg = load_blk(a.gradg + off, blk), y = load_blk(a.Y + off, blk);
        const Blk j = load_blk(a.J + off, blk), bz = load_blk(a.BZ + off, blk);
        Blk gr, r, zero;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            gr.v[i] = gg.v[i] + 0.5f * y.v[i] + 0.5f * rk * (j.v[i] - bz.v[i]);
            r.v[i] = -gr.v[i];
            zero.v[i] = 0.f;
        }
        const Blk z = precond(r, G + (size_t)blk * 4, 0.5f * rk + mu);
        store_blk(a.grad + off, blk, gr);
        store_blk(a.r + off, blk, r);
        store_blk(a.z + off, blk, z);
        store_blk(a.p + off, blk, z);
        store_blk(a.x + off, blk, zero);
        rz += dot_blk(r, z);
    }
    const double rzd = 2.0 * block_sum((double)rz, red);
    if (threadIdx.x == 0) {
        st.rz = rzd;
        st.cg_stop = (rzd > 0.0) ? 0 : 1;
    }
}

// LM bookkeeping of one agent after a residual or trial sweep (modes in LMEvalMode), then the
// PCG initialisation for the next LM step. sm: 2*K*N*4 floats of shared scratch; red: 33 doubles.
__device__ void lm_eval_dev(const LMArgs& a, int agent, int mode, float* sm, double* red) {
    const int N = a.N, K = a.K, KN = K * N;
    const size_t off = (size_t)agent * KN * 8;
    float* Xs = sm;
    float* Gs = sm + KN * 4;
    AgentState& st = a.st[agent];

    if (mode == LM_BEGIN_FROM_PARTIALS) {
        for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) store_blk(a.gradg + off, blk, sum_parts(a, agent, blk, KN));
        __syncthreads();
        project_out_gauge(a.J + off, a.gradg + off, N, K);
        const double pen = block_sum(penalty_part(a.J + off, a.Y + off, a.BZ + off, a.rho, N, KN), red);
        if (threadIdx.x == 0) {
            double g = 0.0;
            for (int ch = 0; ch < a.n_chunks; ++ch) g += a.part_cost[(size_t)agent * a.n_chunks + ch];
            st.g = g;
            st.L = g + pen;
        }
        __syncthreads();
        gram_blocks(a, agent, a.J + off, a.Gm + (size_t)agent * KN * 4, Xs, Gs);
    } else if (mode == LM_BEGIN_REUSE) {
        const double pen = block_sum(penalty_part(a.J + off, a.Y + off, a.BZ + off, a.rho, N, KN), red);
        if (threadIdx.x == 0) st.L = st.g + pen;
        __syncthreads();
    } else {  // LM_ACCEPT: the trial sweep just ran at Jt = J + x
        const double pen_t = block_sum(penalty_part(a.Jt + off, a.Y + off, a.BZ + off, a.rho, N, KN), red);
        const double dpen = block_sum(penalty_decrease_part(a.J + off, a.Jt + off, a.Y + off, a.BZ + off, a.rho, N, KN), red);
        __shared__ int accept_s;
        if (threadIdx.x == 0) {
            double g_t = 0.0, dg = 0.0;
            for (int ch = 0; ch < a.n_chunks; ++ch) {
                if (!a.cost_from_decrease) g_t += __ldcg(a.part_cost + (size_t)agent * a.n_chunks + ch);
                dg += __ldcg(a.part_dcost + (size_t)agent * a.n_chunks + ch);
            }
            if (a.cost_from_decrease) g_t = st.g - dg;
            const double L_t = g_t + pen_t;
            const double dL = dg + dpen;  // L(J) - L(Jt)
            st.g_t = g_t;
            st.L_t = L_t;
            const int acc = (st.pred > 0.0) && isfinite(L_t) && isfinite(dL) && (dL > 0.0);
            if (acc) {
                const double ratio = dL / st.pred;
                const double t = 2.0 * ratio - 1.0;
                st.mu *= fmax(1.0 / 3.0, 1.0 - t * t * t);
                st.nu = 2.0;
                st.g = g_t;
                st.L = L_t;
                st.accepted += 1;
            } else {
                st.mu *= st.nu;
                st.nu *= 2.0;
                st.rejected += 1;
            }
            accept_s = acc;
        }
        __syncthreads();
        if (accept_s) {
            for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
                store_blk(a.gradg + off, blk, sum_parts(a, agent, blk, KN));
                store_blk(a.J + off, blk, load_blk(a.Jt + off, blk));
            }
            __syncthreads();
            project_out_gauge(a.J + off, a.gradg + off, N, K);
            gram_blocks(a, agent, a.J + off, a.Gm + (size_t)agent * KN * 4, Xs, Gs);
        }
    }

    if (mode != LM_ACCEPT) {
        // mu0 = tau * max_{p,k} max diag(G_pk + rho_k/2 I)
        const float* G = a.Gm + (size_t)agent * KN * 4;
        double m = 0.0;
        for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
            const double h = 0.5 * (double)a.rho[blk / N];
            m = fmax(m, fmax((double)G[blk * 4 + 0], (double)G[blk * 4 + 1]) + h);
        }
        m = block_max(m, red);
        if (threadIdx.x == 0) {
            st.mu = a.tau * m;
            st.nu = 2.0;
        }
        __syncthreads();
    }
    cg_init(a, agent, a.Gm + (size_t)agent * KN * 4, red);
}

// One PCG step of one agent after the Hessian sweep of its direction p.
__device__ void cg_step_dev(const LMArgs& a, int agent, double* red) {
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    const int stop = st.cg_stop;
    __syncthreads();
    if (stop) return;
    const float mu = (float)st.mu;
    const double rz = st.rz;
    const float* G = a.Gm + (size_t)agent * KN * 4;

    float pAp_t = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const float lam = 0.5f * a.rho[blk / N] + mu;
        const Blk hp = sum_parts(a, agent, blk, KN);
        const Blk p = load_blk(a.p + off, blk);
        Blk ap;
#pragma unroll
        for (int i = 0; i < 8; ++i) ap.v[i] = hp.v[i] + lam * p.v[i];
        store_blk(a.Ap + off, blk, ap);
        pAp_t += dot_blk(p, ap);
    }
    const double pAp = 2.0 * block_sum((double)pAp_t, red);
    if (!(pAp > 0.0)) {
        if (threadIdx.x == 0) st.cg_stop = 1;
        return;
    }
    const float alpha = (float)(rz / pAp);
    float rzn_t = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const float lam = 0.5f * a.rho[blk / N] + mu;
        Blk x = load_blk(a.x + off, blk), r = load_blk(a.r + off, blk);
        const Blk p = load_blk(a.p + off, blk), ap = load_blk(a.Ap + off, blk);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            x.v[i] = fmaf(alpha, p.v[i], x.v[i]);
            r.v[i] = fmaf(-alpha, ap.v[i], r.v[i]);
        }
        const Blk z = precond(r, G + (size_t)blk * 4, lam);
        store_blk(a.x + off, blk, x);
        store_blk(a.r + off, blk, r);
        store_blk(a.z + off, blk, z);
        rzn_t += dot_blk(r, z);
    }
    const double rzn = 2.0 * block_sum((double)rzn_t, red);
    const float beta = (float)(rzn / rz);
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const Blk z = load_blk(a.z + off, blk);
        Blk p = load_blk(a.p + off, blk);
#pragma unroll
        for (int i = 0; i < 8; ++i) p.v[i] = fmaf(beta, p.v[i], z.v[i]);
        store_blk(a.p + off, blk, p);
    }
    if (threadIdx.x == 0) {
        st.rz = rzn;
        if (!(rzn > 0.0)) st.cg_stop = 1;
    }
}

// Jt = J + x and the predicted decrease of the undamped model.
__device__ void lm_trial_dev(const LMArgs& a, int agent, double* red) {
    const int KN = a.K * a.N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    const double mu = st.mu;
    float xr_t = 0.f, xx_t = 0.f;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const Blk x = load_blk(a.x + off, blk), r = load_blk(a.r + off, blk), gr = load_blk(a.grad + off, blk);
        const Blk j = load_blk(a.J + off, blk);
        Blk jt;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            jt.v[i] = j.v[i] + x.v[i];
            xr_t = fmaf(x.v[i], r.v[i] - gr.v[i], xr_t);
            xx_t = fmaf(x.v[i], x.v[i], xx_t);
        }
        store_blk(a.Jt + off, blk, jt);
    }
    const double xr = block_sum((double)xr_t, red);
    const double xx = block_sum((double)xx_t, red);
    // pred = 1/2 h(x, b + r) + mu/2 h(x, x) with b = -grad, h = 2 * dot
    if (threadIdx.x == 0) st.pred = xr + mu * xx;
}

}  // namespace
}  // namespace calib
