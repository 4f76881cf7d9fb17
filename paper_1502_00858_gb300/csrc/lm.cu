// Per-agent Levenberg-Marquardt / preconditioned-CG kernels of the J-update (Section 3, Eq. M1).
//
// The paper minimises L_i(J, Z^n, Y^n) with Riemannian trust region; this library takes
// n_lm Levenberg-Marquardt steps, each solving the damped Gauss-Newton system
//   (Hess L + mu) x = -grad L,  Hess L = H_GN + rho_k/2 (Eq. HessL),  grad L of Eq. gradL,
// by n_cg preconditioned CG steps from x = 0 with the block-Jacobi preconditioner
// x_pk -> x_pk (G_pk + (rho_k/2 + mu) I)^-1, G_pk the exact (p,k) diagonal block of H_GN.
// Inner products are h(xi, eta) = trace(xi^H eta + eta^H xi) (Eq. inprod) = 2 * (real dot).
// The predicted decrease of the undamped quadratic model is formed without another Hessian pass:
// with b = -grad and the CG residual r = b - (H + rho/2 + mu) x,
//   -h(x, grad) - 1/2 h(x, (H + rho/2) x) = 1/2 h(x, b + r) + mu/2 h(x, x).
// Gain ratio (L(J) - L(J + x)) / pred; accept when pred > 0 and L(J + x) < L(J) (finite). The
// decrease L(J) - L(J + x) is formed directly - the data part by the trial sweep from the model
// change, the penalty part here from x - rather than as a difference of two float32 evaluations
// of L, which near convergence is dominated by round-off.
// Nielsen update mu *= max(1/3, 1 - (2 ratio - 1)^3), nu = 2 on accept, mu *= nu, nu *= 2 on reject.
//
// One CTA per agent. Thread t owns the blocks t, t + T, ... (at most BPT of them, T threads) and
// keeps its share of every vector in registers for the whole kernel, so each kernel reads its
// inputs once and writes its outputs once: the kernels are short chains of dependent global
// loads and block reductions, and their time is latency. Reductions are float32 warp butterflies
// followed by a fixed-order sum of the warp totals (the same value in every thread, no atomics).
#include <math.h>

#include "calib_internal.cuh"
#include "df.cuh"

namespace calib {
namespace {

// At most 512 threads a CTA. With one block per thread (K*N <= 512) at most 64 registers a thread,
// so that 3 agents' CTAs share an SM (320 agents of 320 threads fit 152 SMs in one wave); with two
// (K*N <= 768) at most 384 threads and 80 registers, so that two CTAs share an SM (a few spilled
// bytes cost less than half the resident agents would); larger K*N keeps its blocks in registers.
constexpr int LM_MAX_THREADS = 512;
// Two blocks a thread: at most 384 threads, so that two CTAs share an SM (80 registers a thread).
constexpr int LM_MAX_THREADS_BPT2 = 384;

struct Blk { float v[8]; };

__device__ __forceinline__ Blk ld_blk(const float* base, int blk) {
    const float4* q = reinterpret_cast<const float4*>(base) + 2 * (size_t)blk;
    const float4 a0 = q[0], a1 = q[1];
    return Blk{{a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w}};
}
__device__ __forceinline__ void st_blk(float* base, int blk, const Blk& b) {
    float4* q = reinterpret_cast<float4*>(base) + 2 * (size_t)blk;
    q[0] = make_float4(b.v[0], b.v[1], b.v[2], b.v[3]);
    q[1] = make_float4(b.v[4], b.v[5], b.v[6], b.v[7]);
}
__device__ __forceinline__ Blk zero_blk() { return Blk{{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}}; }
__device__ __forceinline__ float dot8(const Blk& a, const Blk& b) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s = fmaf(a.v[i], b.v[i], s);
    return s;
}

// Sum over the CTA of each v[i]; every thread gets the same totals. red: NV*32 floats owned by
// this call site (no barrier is needed before the next call site writes its own).
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        if (lane == 0) red[i * 32 + w] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float s = 0.f;
        for (int k = 0; k < nw; ++k) s += red[i * 32 + k];
        v[i] = s;
    }
}
__device__ __forceinline__ float block_max(float v, float* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[w] = v;
    __syncthreads();
    float m = red[0];
    for (int k = 1; k < nw; ++k) m = fmaxf(m, red[k]);
    return m;
}
// float64 variant for the values returned to the caller (calib_eval).
__device__ double block_sum_d(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

// x (G + lam I)^-1 for a 2x2 complex block x (row-major re,im pairs) and Hermitian G (g00, g11, re g01, im g01).
__device__ __forceinline__ Blk precond(const Blk& x, const float (&G)[4], float lam) {
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

__device__ __forceinline__ int n_parts(const LMArgs& a, int agent) { return a.part_n ? a.part_n[agent] : a.part_stride; }

// Sum of the partial station sums of a sweep, fixed piece order.
__device__ __forceinline__ Blk sum_parts(const LMArgs& a, int agent, int blk, int KN) {
    const float* base = a.part + (size_t)agent * a.part_stride * KN * 8;
    Blk s = ld_blk(base, blk);
    const int np = n_parts(a, agent);
    for (int ch = 1; ch < np; ++ch) {
        const Blk q = ld_blk(base + (size_t)ch * KN * 8, blk);
#pragma unroll
        for (int i = 0; i < 8; ++i) s.v[i] += q.v[i];
    }
    return s;
}

// Penalty Re tr(Y^H D) + rho/2 ||D||^2 of one block, D = J - BZ (Eq. sumtrace2).
__device__ __forceinline__ float penalty_blk(const Blk& j, const Blk& y, const Blk& bz, float rk) {
    float yd = 0.f, dd = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float d = j.v[i] - bz.v[i];
        yd = fmaf(y.v[i], d, yd);
        dd = fmaf(d, d, dd);
    }
    return yd + 0.5f * rk * dd;
}
// pen(J) - pen(Jt) = -(Re tr(Y^H x) + rho Re tr(D^H x) + rho/2 ||x||^2), D = J - BZ, x = Jt - J, of one
// block. Formed from the small x, so it is accurate relative to the decrease itself.
__device__ __forceinline__ float penalty_decrease_blk(const Blk& j, const Blk& jt, const Blk& y, const Blk& bz, float rk) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float x = jt.v[i] - j.v[i];  // exact: Jt = J + x was rounded once
        const float d = j.v[i] - bz.v[i];
        s -= fmaf(y.v[i], x, rk * fmaf(0.5f * x, x, d * x));
    }
    return s;
}

// ---- gauge projection
// g is invariant under J_k -> J_k U (C = c I_2, Eq. coh), so the exact data gradient has no
// component along the gauge orbit {J_k A : A anti-Hermitian}: the anti-Hermitian part of
// J_k^H G_k vanishes. Float32 residuals leave round-off there, which would otherwise steer the
// weakly determined gauge mode (curved only by the rho/2 penalty). With S = J^H J, solve
// (S A + A S)/2 = skew(J^H G) for A = [[i a, b + i c], [-b + i c, i d]] and set G <- G - J A (the
// h-orthogonal projection); exact arithmetic leaves G unchanged. The skew part is a small
// difference of large station terms, so its sums carry about 48 bits: double-float accumulation
// built from error-free float32 transformations (the exact product error by FMA, Dekker 1971;
// the exact sum error by TwoSum, Knuth TAOCP vol. 2, 4.2.2). The 4x4 system is well conditioned
// (S is the Gram matrix of J_k) and is solved in float32 in closed form.
constexpr int GT = 12;  // per-block gauge terms: 4 double-float (t0, t1, 2 t2, 2 t3) and s0, s1, u, w

// This block's terms of skew(J^H G) and J^H J. Row m, column c of a block: v[m*4 + c*2 + (0 re, 1 im)].
__device__ __forceinline__ void gauge_terms(const Blk& j, const Blk& g, float* out) {
    DF t0{0.f, 0.f}, t1{0.f, 0.f}, t2{0.f, 0.f}, t3{0.f, 0.f};
    float s0 = 0.f, s1 = 0.f, u = 0.f, w = 0.f;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const float a0r = j.v[m * 4 + 0], a0i = j.v[m * 4 + 1], a1r = j.v[m * 4 + 2], a1i = j.v[m * 4 + 3];
        const float g0r = g.v[m * 4 + 0], g0i = g.v[m * 4 + 1], g1r = g.v[m * 4 + 2], g1i = g.v[m * 4 + 3];
        // t0 = Im M00, t1 = Im M11 with M = J^H G
        df_add_prod(t0, a0r, g0i);
        df_add_prod(t0, -a0i, g0r);
        df_add_prod(t1, a1r, g1i);
        df_add_prod(t1, -a1i, g1r);
        // 2 t2 = Re M01 - Re M10,  2 t3 = Im M01 + Im M10
        df_add_prod(t2, a0r, g1r);
        df_add_prod(t2, a0i, g1i);
        df_add_prod(t2, -a1r, g0r);
        df_add_prod(t2, -a1i, g0i);
        df_add_prod(t3, a0r, g1i);
        df_add_prod(t3, -a0i, g1r);
        df_add_prod(t3, a1r, g0i);
        df_add_prod(t3, -a1i, g0r);
        s0 = fmaf(a0r, a0r, fmaf(a0i, a0i, s0));
        s1 = fmaf(a1r, a1r, fmaf(a1i, a1i, s1));
        u = fmaf(a0r, a1r, fmaf(a0i, a1i, u));
        w = fmaf(a0r, a1i, fmaf(-a0i, a1r, w));
    }
    out[0] = t0.hi; out[1] = t0.lo; out[2] = t1.hi; out[3] = t1.lo;
    out[4] = t2.hi; out[5] = t2.lo; out[6] = t3.hi; out[7] = t3.lo;
    out[8] = s0; out[9] = s1; out[10] = u; out[11] = w;
}

// Solve the gauge system of one direction from its summed terms; A = (a, d, b, c).
// Eliminating b and c (rows 3 and 4) leaves two scalar equations in a and d whose sum gives
// e = a + d with the determinant of S as denominator.
__device__ __forceinline__ float4 gauge_solve(const float (&tt)[GT]) {
    const float t0 = tt[0] + tt[1], t1 = tt[2] + tt[3], T2 = tt[4] + tt[5], T3 = tt[6] + tt[7];
    const float s0 = tt[8], s1 = tt[9], u = tt[10], w = tt[11];
    const float sig = s0 + s1, uw = u * u + w * w;
    const float det = s0 * s1 - uw;
    if (!(sig > 0.f) || !(det > 1e-12f * sig * sig) || !isfinite(T2 + T3 + t0 + t1)) return make_float4(0.f, 0.f, 0.f, 0.f);
    const float h = (u * T3 - w * T2) / sig, q = uw / sig;
    const float e = ((t0 - h) * s1 + (t1 - h) * s0) / det;
    return make_float4((t0 - h + q * e) / s0, (t1 - h + q * e) / s1, (T2 + w * e) / sig, (T3 - u * e) / sig);
}

// Project the gauge component out of this CTA's data-gradient blocks g (held by their threads).
// sm: KN*GT floats; Asol: 4*K floats.
template <int BPT>
__device__ void project_out_gauge(const Blk (&j)[BPT], Blk (&g)[BPT], int K, int N, float* sm, float* Asol) {
    const int T = blockDim.x, KN = K * N;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = threadIdx.x + i * T;
        if (blk < KN) gauge_terms(j[i], g[i], sm + (size_t)blk * GT);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
    for (int k = warp; k < K; k += nw) {
        DF t[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = lane; p < N; p += 32) {
            const float* q = sm + (size_t)(k * N + p) * GT;
#pragma unroll
            for (int i = 0; i < 4; ++i) t[i] = df_add(t[i], DF{q[2 * i], q[2 * i + 1]});
#pragma unroll
            for (int i = 0; i < 4; ++i) s[i] += q[8 + i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const DF other{__shfl_xor_sync(0xffffffffu, t[i].hi, o), __shfl_xor_sync(0xffffffffu, t[i].lo, o)};
                t[i] = df_add(t[i], other);
                s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
            }
        }
        if (lane == 0) {
            const float tt[GT] = {t[0].hi, t[0].lo, t[1].hi, t[1].lo, t[2].hi, t[2].lo, t[3].hi, t[3].lo,
                                  s[0], s[1], s[2], s[3]};
            const float4 A = gauge_solve(tt);
            Asol[k * 4 + 0] = A.x;
            Asol[k * 4 + 1] = A.y;
            Asol[k * 4 + 2] = A.z;
            Asol[k * 4 + 3] = A.w;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = threadIdx.x + i * T;
        if (blk >= KN) continue;
        const int k = blk / N;
        const float a = Asol[k * 4 + 0], d = Asol[k * 4 + 1], b = Asol[k * 4 + 2], c = Asol[k * 4 + 3];
        // A = [[i a, b + i c], [-b + i c, i d]]
        const float A00r = 0.f, A00i = a, A01r = b, A01i = c, A10r = -b, A10i = c, A11r = 0.f, A11i = d;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float jr0 = j[i].v[r * 4 + 0], ji0 = j[i].v[r * 4 + 1], jr1 = j[i].v[r * 4 + 2], ji1 = j[i].v[r * 4 + 3];
            // (J A)[r][0] = J[r][0] A00 + J[r][1] A10 ; (J A)[r][1] = J[r][0] A01 + J[r][1] A11
            g[i].v[r * 4 + 0] -= jr0 * A00r - ji0 * A00i + jr1 * A10r - ji1 * A10i;
            g[i].v[r * 4 + 1] -= jr0 * A00i + ji0 * A00r + jr1 * A10i + ji1 * A10r;
            g[i].v[r * 4 + 2] -= jr0 * A01r - ji0 * A01i + jr1 * A11r - ji1 * A11i;
            g[i].v[r * 4 + 3] -= jr0 * A01i + ji0 * A01r + jr1 * A11i + ji1 * A11r;
        }
    }
}

// Jacobi blocks G_pk = sum_o s_(p,o)k J_ok^H J_ok at the CTA's J (held by the threads), from the
// dense weights gw (thread (k, p) reads its 16-byte aligned row, all loads independent) and the
// products J_ok^H J_ok staged in sm (KN*4 floats).
template <int BPT>
__device__ void gram_blocks(const LMArgs& a, int agent, const Blk (&j)[BPT], float* sm, float (&G)[BPT][4]) {
    const int T = blockDim.x, N = a.N, K = a.K, KN = K * N;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = threadIdx.x + i * T;
        if (blk >= KN) continue;
        const float* v = j[i].v;
        // J^H J: x00 = |J00|^2 + |J10|^2, x11 = |J01|^2 + |J11|^2, x01 = conj(J00) J01 + conj(J10) J11
        reinterpret_cast<float4*>(sm)[blk] = make_float4(
            v[0] * v[0] + v[1] * v[1] + v[4] * v[4] + v[5] * v[5],
            v[2] * v[2] + v[3] * v[3] + v[6] * v[6] + v[7] * v[7],
            v[0] * v[2] + v[1] * v[3] + v[4] * v[6] + v[5] * v[7],
            v[0] * v[3] - v[1] * v[2] + v[4] * v[7] - v[5] * v[6]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = threadIdx.x + i * T;
        G[i][0] = G[i][1] = G[i][2] = G[i][3] = 0.f;
        if (blk >= KN) continue;
        const int k = blk / N, p = blk - k * N;
        const int NW4 = (N + 3) / 4;
        const float4* W = reinterpret_cast<const float4*>(a.gw + (((size_t)agent * K + k) * N + p) * NW4 * 4);
        const float4* X = reinterpret_cast<const float4*>(sm) + k * N;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll 16
        for (int o4 = 0; o4 < NW4; ++o4) {
            const float4 w4 = __ldg(W + o4);
            const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = 4 * o4 + q;
                if (o >= N) break;  // row padding
                const float4 x = X[o];
                g0 = fmaf(wv[q], x.x, g0);
                g1 = fmaf(wv[q], x.y, g1);
                g2 = fmaf(wv[q], x.z, g2);
                g3 = fmaf(wv[q], x.w, g3);
            }
        }
        G[i][0] = g0; G[i][1] = g1; G[i][2] = g2; G[i][3] = g3;
        reinterpret_cast<float4*>(a.Gm + (size_t)agent * KN * 4)[blk] = make_float4(g0, g1, g2, g3);
    }
}

// ---- kernels

// LM bookkeeping of one agent after a residual or trial sweep (modes in LMEvalMode), then the
// PCG initialisation for the next LM step: grad = gradg + Y/2 + rho/2 (J - BZ), r = -grad,
// p = z = M^-1 r, x = 0, rz = h(r, z).
template <int BPT>
__global__ void __launch_bounds__(BPT == 2 ? LM_MAX_THREADS_BPT2 : LM_MAX_THREADS, BPT <= 2 ? 2 : 1) k_lm_eval(const LMArgs a, const int mode) {
    extern __shared__ __align__(16) float sm[];  // KN*GT floats (gauge terms), reused for J^H J
    __shared__ float red[4][64];
    __shared__ float Asol[MAX_K * 4];
    __shared__ int accept_s;
    __shared__ float mu_s;
    const int agent = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int N = a.N, K = a.K, KN = K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];

    // J, Y, BZ and J' are read before the dependency wait: the preceding kernel (a residual or
    // trial sweep, or the fusion-centre step's record kernel) writes only partials and records.
    Blk j[BPT], y[BPT], bz[BPT], gg[BPT], jt[BPT];
    float rk[BPT];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        j[i] = y[i] = bz[i] = gg[i] = jt[i] = zero_blk();
        rk[i] = 0.f;
        if (blk < KN) {
            j[i] = ld_blk(a.J + off, blk);
            y[i] = ld_blk(a.Y + off, blk);
            bz[i] = ld_blk(a.BZ + off, blk);
            if (mode == LM_ACCEPT) jt[i] = ld_blk(a.Jt + off, blk);
            rk[i] = a.rho[blk / N];
        }
    }
    griddep_wait();
    griddep_launch_dependents();
    bool fresh = false;  // gradg re-formed from the sweep's partials: project it and rebuild G
    if (mode == LM_ACCEPT) {  // the trial sweep just ran at Jt = J + x
        float v[2] = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk < KN) {
                v[0] += penalty_blk(jt[i], y[i], bz[i], rk[i]);
                v[1] += penalty_decrease_blk(j[i], jt[i], y[i], bz[i], rk[i]);
            }
        }
        block_sum<2>(v, red[0]);
        if (tid == 0) {
            double g_t = 0.0, dg = 0.0;
            const int np = n_parts(a, agent);
            for (int ch = 0; ch < np; ++ch) {
                if (!a.cost_from_decrease) g_t += a.part_cost[(size_t)agent * a.part_stride + ch];
                dg += a.part_dcost[(size_t)agent * a.part_stride + ch];
            }
            if (a.cost_from_decrease) g_t = st.g - dg;
            const double L_t = g_t + (double)v[0];
            const double dL = dg + (double)v[1];  // L(J) - L(Jt)
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
            mu_s = (float)st.mu;
        }
        __syncthreads();
        fresh = accept_s != 0;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            if (fresh) {
                j[i] = jt[i];
                st_blk(a.J + off, blk, j[i]);
                gg[i] = sum_parts(a, agent, blk, KN);
            } else {
                gg[i] = ld_blk(a.gradg + off, blk);
            }
        }
    } else {
        float v[1] = {0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            gg[i] = (mode == LM_BEGIN_FROM_PARTIALS) ? sum_parts(a, agent, blk, KN) : ld_blk(a.gradg + off, blk);
            v[0] += penalty_blk(j[i], y[i], bz[i], rk[i]);
        }
        block_sum<1>(v, red[0]);
        if (tid == 0) {
            if (mode == LM_BEGIN_FROM_PARTIALS) {
                double g = 0.0;
                for (int ch = 0; ch < n_parts(a, agent); ++ch) g += a.part_cost[(size_t)agent * a.part_stride + ch];
                st.g = g;
            }
            st.L = st.g + (double)v[0];
        }
        fresh = mode == LM_BEGIN_FROM_PARTIALS;
    }

    float G[BPT][4];
    if (fresh) {
        project_out_gauge<BPT>(j, gg, K, N, sm, Asol);
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk < KN) st_blk(a.gradg + off, blk, gg[i]);
        }
        __syncthreads();  // sm is reused for J^H J
        gram_blocks<BPT>(a, agent, j, sm, G);
    } else {
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            G[i][0] = G[i][1] = G[i][2] = G[i][3] = 0.f;
            if (blk < KN) {
                const float4 q = reinterpret_cast<const float4*>(a.Gm + (size_t)agent * KN * 4)[blk];
                G[i][0] = q.x; G[i][1] = q.y; G[i][2] = q.z; G[i][3] = q.w;
            }
        }
    }
    if (mode != LM_ACCEPT) {
        // mu0 = tau * max_{p,k} max diag(G_pk + rho_k/2 I)
        float m = 0.f;
#pragma unroll
        for (int i = 0; i < BPT; ++i)
            if (tid + i * T < KN) m = fmaxf(m, fmaxf(G[i][0], G[i][1]) + 0.5f * rk[i]);
        m = block_max(m, red[1]);
        if (tid == 0) {
            st.mu = a.tau * (double)m;
            st.nu = 2.0;
            mu_s = (float)st.mu;
        }
        __syncthreads();
    }
    const float mu = mu_s;
    float rz[1] = {0.f};
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        if (blk >= KN) continue;
        Blk gr, r;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            gr.v[e] = gg[i].v[e] + 0.5f * y[i].v[e] + 0.5f * rk[i] * (j[i].v[e] - bz[i].v[e]);
            r.v[e] = -gr.v[e];
        }
        const Blk z = precond(r, G[i], 0.5f * rk[i] + mu);
        st_blk(a.grad + off, blk, gr);
        st_blk(a.r + off, blk, r);
        st_blk(a.p + off, blk, z);
        st_blk(a.x + off, blk, zero_blk());
        rz[0] += dot8(r, z);
    }
    block_sum<1>(rz, red[2]);
    if (tid == 0) {
        const double rzd = 2.0 * (double)rz[0];
        st.rz = rzd;
        st.cg_stop = (rzd > 0.0) ? 0 : 1;
    }
}

// One PCG step of one agent after the Hessian sweep of its direction p; with last set, also the
// LM trial point Jt = J + x and the predicted decrease pred = 1/2 h(x, b + r) + mu/2 h(x, x).
template <int BPT>
__global__ void __launch_bounds__(BPT == 2 ? LM_MAX_THREADS_BPT2 : LM_MAX_THREADS, BPT <= 2 ? 2 : 1) k_cg_step(const LMArgs a, const int last) {
    __shared__ float red[3][64];
    const int agent = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    // Every load first, independent of the stop flag, so that they are in flight together. The
    // preceding kernel is the Hessian pass, which writes only the partials: the PCG vectors, the
    // Jacobi blocks and the agent state are read before the dependency wait.
    Blk x[BPT], r[BPT], p[BPT], ap[BPT];  // ap holds the Hessian partial sum until it becomes A p
    float lam[BPT], G[BPT][4];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        x[i] = r[i] = p[i] = ap[i] = zero_blk();
        lam[i] = 0.f;
        G[i][0] = G[i][1] = G[i][2] = G[i][3] = 0.f;
        if (blk >= KN) continue;
        x[i] = ld_blk(a.x + off, blk);
        r[i] = ld_blk(a.r + off, blk);
        p[i] = ld_blk(a.p + off, blk);
        const float4 q = reinterpret_cast<const float4*>(a.Gm + (size_t)agent * KN * 4)[blk];
        G[i][0] = q.x; G[i][1] = q.y; G[i][2] = q.z; G[i][3] = q.w;
        lam[i] = 0.5f * a.rho[blk / N];
    }
    const int stop = a.timing ? 0 : st.cg_stop;
    const float mu = a.timing ? 1.f : (float)st.mu;
    const float rz = a.timing ? 1.f : (float)st.rz;
    griddep_wait();
    griddep_launch_dependents();
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        if (blk < KN) ap[i] = sum_parts(a, agent, blk, KN);
    }
    if (!stop) {
        float v[1] = {0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            lam[i] += mu;
#pragma unroll
            for (int e = 0; e < 8; ++e) ap[i].v[e] = fmaf(lam[i], p[i].v[e], ap[i].v[e]);
            v[0] += dot8(p[i], ap[i]);
        }
        block_sum<1>(v, red[0]);
        const float pAp = 2.f * v[0];
        if (pAp > 0.f || a.timing) {  // the same value in every thread
            const float alpha = rz / pAp;
            float w[1] = {0.f};
#pragma unroll
            for (int i = 0; i < BPT; ++i) {
                if (tid + i * T >= KN) continue;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    x[i].v[e] = fmaf(alpha, p[i].v[e], x[i].v[e]);
                    r[i].v[e] = fmaf(-alpha, ap[i].v[e], r[i].v[e]);
                }
                ap[i] = precond(r[i], G[i], lam[i]);  // z
                w[0] += dot8(r[i], ap[i]);
            }
            block_sum<1>(w, red[1]);
            const float rzn = 2.f * w[0];
            const float beta = rzn / rz;
#pragma unroll
            for (int i = 0; i < BPT; ++i) {
                const int blk = tid + i * T;
                if (blk >= KN) continue;
#pragma unroll
                for (int e = 0; e < 8; ++e) p[i].v[e] = fmaf(beta, p[i].v[e], ap[i].v[e]);
                st_blk(a.x + off, blk, x[i]);
                st_blk(a.r + off, blk, r[i]);
                st_blk(a.p + off, blk, p[i]);
            }
            if (tid == 0 && !a.timing) {
                st.rz = (double)rzn;
                if (!(rzn > 0.f)) st.cg_stop = 1;
            }
        } else if (tid == 0) {
            st.cg_stop = 1;
        }
    }
    if (last) {
        float v[2] = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            const Blk jb = ld_blk(a.J + off, blk), gr = ld_blk(a.grad + off, blk);
            Blk jt;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                jt.v[e] = jb.v[e] + x[i].v[e];
                v[0] = fmaf(x[i].v[e], r[i].v[e] - gr.v[e], v[0]);
                v[1] = fmaf(x[i].v[e], x[i].v[e], v[1]);
            }
            st_blk(a.Jt + off, blk, jt);
        }
        block_sum<2>(v, red[2]);
        // pred = 1/2 h(x, b + r) + mu/2 h(x, x) with b = -grad, h = 2 * dot
        if (tid == 0) st.pred = (double)v[0] + st.mu * (double)v[1];
    }
}

// ---- Riemannian trust region (the paper's inner solver for Eq. M1, Section 3 and Appendix A)
//
// In Euclidean space the retraction is J + eta and the Riemannian gradient and Hessian are grad L
// (Eq. gradL) and Hess L (Eq. HessL, Gauss-Newton part), so one RTR step is: truncated CG
// (Steihaug-Toint, no preconditioner, norm ||x||_h = sqrt(h(x, x))) on the model
// m(eta) = h(grad, eta) + 1/2 h(eta, Hess L[eta]) within the radius Delta, then the ratio
// rho = (L(J) - L(J + eta)) / (m(0) - m(eta)) decides the step and the radius (Absil, Baker and
// Gallivan 2007): accept when rho > 0.1; Delta /= 4 when rho < 1/4; Delta = min(2 Delta, Delta_bar)
// when rho > 3/4 and the CG stopped on the boundary. Delta_bar = ||J0||_h at the start of the
// J-update, Delta_0 = Delta_bar / 8. The CG stops on the boundary, on non-positive curvature
// (both then step to the boundary along d), when ||r|| <= ||r0|| min(||r0||, 0.1), or after n_cg
// steps. Sign convention as in PCG: r = b - Hess L[eta] with b = -grad, d_0 = r_0, so the model
// decrease is m(0) - m(eta) = 1/2 h(eta, b + r), formed from the CG residual without another sweep.
constexpr double TCG_KAPPA = 0.1;   // residual test ||r|| <= ||r0|| min(||r0||, kappa)
constexpr double RTR_ACCEPT = 0.1;  // a step is accepted when its ratio exceeds this

// One truncated-CG step of one agent after the Hessian sweep of its direction d (in a.p); with
// last set, also J' = J + eta and the predicted decrease 1/2 h(eta, b + r).
template <int BPT>
__global__ void __launch_bounds__(BPT == 2 ? LM_MAX_THREADS_BPT2 : LM_MAX_THREADS, BPT <= 2 ? 2 : 1) k_tcg_step(const LMArgs a, const int last) {
    // one area per reduction call site (block_sum<NV> uses NV * 32 floats)
    __shared__ float red_d[3 * 32], red_r[32], red_p[32];
    const int agent = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    Blk x[BPT], r[BPT], p[BPT], ap[BPT];  // eta, r, d; ap: the Hessian partial sum, then Hess L[d]
    float lam[BPT];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        x[i] = r[i] = p[i] = ap[i] = zero_blk();
        lam[i] = 0.f;
        if (blk >= KN) continue;
        x[i] = ld_blk(a.x + off, blk);
        r[i] = ld_blk(a.r + off, blk);
        p[i] = ld_blk(a.p + off, blk);
        ap[i] = sum_parts(a, agent, blk, KN);
        lam[i] = 0.5f * a.rho[blk / N];
    }
    // the agent's scalars, read before any thread can write them
    const int stop = st.cg_stop;
    const double rr = st.rz, ee = st.ee, delta = st.delta, r0sq = st.r0sq;
    if (stop == TCG_RUNNING) {
        float v[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            if (tid + i * T >= KN) continue;
#pragma unroll
            for (int e = 0; e < 8; ++e) ap[i].v[e] = fmaf(lam[i], p[i].v[e], ap[i].v[e]);
            v[0] += dot8(p[i], ap[i]);
            v[1] += dot8(x[i], p[i]);
            v[2] += dot8(p[i], p[i]);
        }
        block_sum<3>(v, red_d);
        const double dHd = 2.0 * v[0], ed = 2.0 * v[1], dd = 2.0 * v[2];  // h(d, Hd), h(eta, d), h(d, d)
        int why = TCG_RUNNING;
        double step = 0.0, ee_new = ee;
        if (!(dHd > 0.0)) {
            why = TCG_CURVATURE;
        } else {
            step = rr / dHd;
            ee_new = ee + 2.0 * step * ed + step * step * dd;
            if (ee_new >= delta * delta) why = TCG_BOUNDARY;
        }
        if (why != TCG_RUNNING) {  // to the boundary along d: ||eta + tau d||_h = Delta, tau >= 0
            step = (dd > 0.0) ? (-ed + sqrt(fmax(ed * ed + dd * (delta * delta - ee), 0.0))) / dd : 0.0;
            ee_new = delta * delta;
        }
        const float sf = (float)step;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            if (tid + i * T >= KN) continue;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                x[i].v[e] = fmaf(sf, p[i].v[e], x[i].v[e]);
                r[i].v[e] = fmaf(-sf, ap[i].v[e], r[i].v[e]);
            }
        }
        double rr_new = rr;
        if (why == TCG_RUNNING) {
            float w[1] = {0.f};
#pragma unroll
            for (int i = 0; i < BPT; ++i)
                if (tid + i * T < KN) w[0] += dot8(r[i], r[i]);
            block_sum<1>(w, red_r);
            rr_new = 2.0 * w[0];
            if (rr_new <= r0sq * fmin(r0sq, TCG_KAPPA * TCG_KAPPA)) {
                why = TCG_RESIDUAL;
            } else {
                const float beta = (float)(rr_new / rr);
#pragma unroll
                for (int i = 0; i < BPT; ++i) {
                    if (tid + i * T >= KN) continue;
#pragma unroll
                    for (int e = 0; e < 8; ++e) p[i].v[e] = fmaf(beta, p[i].v[e], r[i].v[e]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            st_blk(a.x + off, blk, x[i]);
            st_blk(a.r + off, blk, r[i]);
            st_blk(a.p + off, blk, p[i]);
        }
        if (tid == 0) {
            st.rz = rr_new;
            st.ee = ee_new;
            st.cg_stop = why;
        }
    }
    if (last) {
        float v[1] = {0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            const Blk jb = ld_blk(a.J + off, blk), gr = ld_blk(a.grad + off, blk);
            Blk jt;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                jt.v[e] = jb.v[e] + x[i].v[e];
                v[0] = fmaf(x[i].v[e], r[i].v[e] - gr.v[e], v[0]);
            }
            st_blk(a.Jt + off, blk, jt);
        }
        block_sum<1>(v, red_p);
        if (tid == 0) st.pred = (double)v[0];  // 1/2 h(eta, b + r), h = 2 * dot
    }
}

// Trust-region bookkeeping of one agent after a residual or trial sweep (modes in LMEvalMode), then
// the start of the next truncated CG: grad = gradg + Y/2 + rho/2 (J - BZ), r = d = -grad, eta = 0.
// The begin modes set Delta_bar = ||J||_h and Delta = Delta_bar / 8.
template <int BPT>
__global__ void __launch_bounds__(BPT == 2 ? LM_MAX_THREADS_BPT2 : LM_MAX_THREADS, BPT <= 2 ? 2 : 1) k_rtr_eval(const LMArgs a, const int mode) {
    extern __shared__ __align__(16) float sm[];  // KN*GT floats (gauge terms)
    __shared__ float red[4][64];
    __shared__ float Asol[MAX_K * 4];
    __shared__ int accept_s;
    const int agent = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int N = a.N, K = a.K, KN = K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];

    Blk j[BPT], y[BPT], bz[BPT], gg[BPT];
    float rk[BPT];
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        j[i] = y[i] = bz[i] = gg[i] = zero_blk();
        rk[i] = 0.f;
        if (blk < KN) {
            j[i] = ld_blk(a.J + off, blk);
            y[i] = ld_blk(a.Y + off, blk);
            bz[i] = ld_blk(a.BZ + off, blk);
            rk[i] = a.rho[blk / N];
        }
    }
    bool fresh = false;
    if (mode == LM_ACCEPT) {  // the trial sweep just ran at J' = J + eta
        Blk jt[BPT];
        float v[2] = {0.f, 0.f};
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            jt[i] = zero_blk();
            if (blk < KN) {
                jt[i] = ld_blk(a.Jt + off, blk);
                v[0] += penalty_blk(jt[i], y[i], bz[i], rk[i]);
                v[1] += penalty_decrease_blk(j[i], jt[i], y[i], bz[i], rk[i]);
            }
        }
        block_sum<2>(v, red[0]);
        if (tid == 0) {
            double g_t = 0.0, dg = 0.0;
            const int np = n_parts(a, agent);
            for (int ch = 0; ch < np; ++ch) {
                if (!a.cost_from_decrease) g_t += a.part_cost[(size_t)agent * a.part_stride + ch];
                dg += a.part_dcost[(size_t)agent * a.part_stride + ch];
            }
            if (a.cost_from_decrease) g_t = st.g - dg;
            const double L_t = g_t + (double)v[0];
            const double dL = dg + (double)v[1];  // L(J) - L(J')
            st.g_t = g_t;
            st.L_t = L_t;
            const double ratio = (st.pred > 0.0 && isfinite(L_t) && isfinite(dL)) ? dL / st.pred : -INFINITY;
            if (ratio < 0.25)
                st.delta *= 0.25;
            else if (ratio > 0.75 && (st.cg_stop == TCG_BOUNDARY || st.cg_stop == TCG_CURVATURE))
                st.delta = fmin(2.0 * st.delta, st.delta_bar);
            const int acc = ratio > RTR_ACCEPT;
            if (acc) {
                st.g = g_t;
                st.L = L_t;
                st.accepted += 1;
            } else {
                st.rejected += 1;
            }
            accept_s = acc;
        }
        __syncthreads();
        fresh = accept_s != 0;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            if (fresh) {
                j[i] = jt[i];
                st_blk(a.J + off, blk, j[i]);
                gg[i] = sum_parts(a, agent, blk, KN);
            } else {
                gg[i] = ld_blk(a.gradg + off, blk);
            }
        }
    } else {
        float v[2] = {0.f, 0.f};  // penalty, ||J||^2
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk >= KN) continue;
            gg[i] = (mode == LM_BEGIN_FROM_PARTIALS || mode == LM_BEGIN_FROM_TRIAL) ? sum_parts(a, agent, blk, KN)
                                                                                 : ld_blk(a.gradg + off, blk);
            v[0] += penalty_blk(j[i], y[i], bz[i], rk[i]);
            v[1] += dot8(j[i], j[i]);
        }
        block_sum<2>(v, red[0]);
        if (tid == 0) {
            if (mode == LM_BEGIN_FROM_PARTIALS) {
                double g = 0.0;
                for (int ch = 0; ch < n_parts(a, agent); ++ch) g += a.part_cost[(size_t)agent * a.part_stride + ch];
                st.g = g;
            } else if (mode == LM_BEGIN_FROM_TRIAL) {
                st.g = 0.0;  // costs of this sub-problem are tracked relative to its start
            }
            st.L = st.g + (double)v[0];
            st.delta_bar = sqrt(2.0 * (double)v[1]);
            st.delta = st.delta_bar / 8.0;
        }
        fresh = mode == LM_BEGIN_FROM_PARTIALS || mode == LM_BEGIN_FROM_TRIAL;
    }
    if (fresh) {
        project_out_gauge<BPT>(j, gg, K, N, sm, Asol);
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int blk = tid + i * T;
            if (blk < KN) st_blk(a.gradg + off, blk, gg[i]);
        }
    }
    float rr[1] = {0.f};
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        const int blk = tid + i * T;
        if (blk >= KN) continue;
        Blk gr, r;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            gr.v[e] = gg[i].v[e] + 0.5f * y[i].v[e] + 0.5f * rk[i] * (j[i].v[e] - bz[i].v[e]);
            r.v[e] = -gr.v[e];
        }
        st_blk(a.grad + off, blk, gr);
        st_blk(a.r + off, blk, r);
        st_blk(a.p + off, blk, r);
        st_blk(a.x + off, blk, zero_blk());
        rr[0] += dot8(r, r);
    }
    block_sum<1>(rr, red[2]);
    if (tid == 0) {
        const double h = 2.0 * (double)rr[0];
        st.rz = h;
        st.r0sq = h;
        st.ee = 0.0;
        st.cg_stop = (h > 0.0) ? TCG_RUNNING : TCG_RESIDUAL;
    }
}

// calib_eval: L, g and grad L at a given J (sweep already ran on J), without touching the state.
__global__ void __launch_bounds__(256) k_eval_output(const LMArgs a, float* grad_out, double* L_out, double* g_out) {
    __shared__ double red[32];
    const int agent = blockIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    double pen = 0.0;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const double rk = a.rho[blk / N];
        const Blk gg = sum_parts(a, agent, blk, KN);
        const Blk y = ld_blk(a.Y + off, blk), j = ld_blk(a.Jt + off, blk), bz = ld_blk(a.BZ + off, blk);
        Blk gr;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const double d = (double)j.v[i] - (double)bz.v[i];
            gr.v[i] = (float)((double)gg.v[i] + 0.5 * (double)y.v[i] + 0.5 * rk * d);
            pen += (double)y.v[i] * d + 0.5 * rk * d * d;
        }
        st_blk(grad_out + off, blk, gr);
    }
    pen = block_sum_d(pen, red);
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int ch = 0; ch < n_parts(a, agent); ++ch) g += a.part_cost[(size_t)agent * a.part_stride + ch];
        if (g_out) g_out[agent] = g;
        if (L_out) L_out[agent] = g + pen;
    }
}

// calib_hessvec: out = H_GN eta + rho/2 eta (eta passed in a.p).
__global__ void __launch_bounds__(256) k_hv_output(const LMArgs a, float* out) {
    const int agent = blockIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const float h = 0.5f * a.rho[blk / N];
        const Blk hp = sum_parts(a, agent, blk, KN);
        const Blk e = ld_blk(a.p + off, blk);
        Blk o;
#pragma unroll
        for (int i = 0; i < 8; ++i) o.v[i] = hp.v[i] + h * e.v[i];
        st_blk(out + off, blk, o);
    }
}

// Blocks per thread and threads per CTA for K*N blocks.
struct LMShape { int bpt, threads; };
LMShape lm_shape(int KN) {
    int bpt = 1;
    while ((KN + bpt - 1) / bpt > (bpt == 2 ? LM_MAX_THREADS_BPT2 : LM_MAX_THREADS)) bpt *= 2;
    const int t = (KN + bpt - 1) / bpt;
    return LMShape{bpt, ((t + 31) / 32) * 32};
}

template <int BPT>
cudaError_t eval_go(const LMArgs& a, int mode, int threads, cudaStream_t s) {
    const size_t smem = (size_t)a.K * a.N * GT * sizeof(float);
    return launch_k(a.pdl != 0, k_lm_eval<BPT>, a.A, threads, smem, s, a, mode);
}
template <int BPT>
cudaError_t cg_go(const LMArgs& a, bool last, int threads, cudaStream_t s) {
    return launch_k(a.pdl != 0, k_cg_step<BPT>, a.A, threads, 0, s, a, last ? 1 : 0);
}
template <int BPT>
cudaError_t rtr_eval_go(const LMArgs& a, int mode, int threads, cudaStream_t s) {
    const size_t smem = (size_t)a.K * a.N * GT * sizeof(float);
    k_rtr_eval<BPT><<<a.A, threads, smem, s>>>(a, mode);
    return cudaGetLastError();
}
template <int BPT>
cudaError_t tcg_go(const LMArgs& a, bool last, int threads, cudaStream_t s) {
    k_tcg_step<BPT><<<a.A, threads, 0, s>>>(a, last ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t prepare_lm_kernels() {
    const int smem = MAX_K * MAX_N * GT * (int)sizeof(float) > 200 * 1024 ? 200 * 1024 : MAX_K * MAX_N * GT * (int)sizeof(float);
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_lm_eval<1>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_lm_eval<2>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_lm_eval<4>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_lm_eval<8>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rtr_eval<1>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rtr_eval<2>, attr, smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rtr_eval<4>, attr, smem)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rtr_eval<8>, attr, smem);
}

cudaError_t launch_lm_eval(const LMArgs& a, int mode, cudaStream_t s) {
    const LMShape sh = lm_shape(a.K * a.N);
    if ((size_t)a.K * a.N * GT * sizeof(float) > 200 * 1024) return cudaErrorInvalidConfiguration;
    switch (sh.bpt) {
        case 1: return eval_go<1>(a, mode, sh.threads, s);
        case 2: return eval_go<2>(a, mode, sh.threads, s);
        case 4: return eval_go<4>(a, mode, sh.threads, s);
        case 8: return eval_go<8>(a, mode, sh.threads, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
cudaError_t launch_cg_step(const LMArgs& a, bool last, cudaStream_t s) {
    const LMShape sh = lm_shape(a.K * a.N);
    switch (sh.bpt) {
        case 1: return cg_go<1>(a, last, sh.threads, s);
        case 2: return cg_go<2>(a, last, sh.threads, s);
        case 4: return cg_go<4>(a, last, sh.threads, s);
        case 8: return cg_go<8>(a, last, sh.threads, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
cudaError_t launch_rtr_eval(const LMArgs& a, int mode, cudaStream_t s) {
    const LMShape sh = lm_shape(a.K * a.N);
    if ((size_t)a.K * a.N * GT * sizeof(float) > 200 * 1024) return cudaErrorInvalidConfiguration;
    switch (sh.bpt) {
        case 1: return rtr_eval_go<1>(a, mode, sh.threads, s);
        case 2: return rtr_eval_go<2>(a, mode, sh.threads, s);
        case 4: return rtr_eval_go<4>(a, mode, sh.threads, s);
        case 8: return rtr_eval_go<8>(a, mode, sh.threads, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
cudaError_t launch_tcg_step(const LMArgs& a, bool last, cudaStream_t s) {
    const LMShape sh = lm_shape(a.K * a.N);
    switch (sh.bpt) {
        case 1: return tcg_go<1>(a, last, sh.threads, s);
        case 2: return tcg_go<2>(a, last, sh.threads, s);
        case 4: return tcg_go<4>(a, last, sh.threads, s);
        case 8: return tcg_go<8>(a, last, sh.threads, s);
        default: return cudaErrorInvalidConfiguration;
    }
}
cudaError_t launch_eval_output(const LMArgs& a, float* grad_out, double* L_out, double* g_out, cudaStream_t s) {
    k_eval_output<<<a.A, 256, 0, s>>>(a, grad_out, L_out, g_out);
    return cudaGetLastError();
}
cudaError_t launch_hv_output(const LMArgs& a, float* out, cudaStream_t s) {
    k_hv_output<<<a.A, 256, 0, s>>>(a, out);
    return cudaGetLastError();
}

}  // namespace calib
