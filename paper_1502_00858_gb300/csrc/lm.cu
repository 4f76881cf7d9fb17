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
// change, the penalty part here in float64 from x - rather than as a difference of two float32
// evaluations of L, which near convergence is dominated by round-off.
// Nielsen update mu *= max(1/3, 1 - (2 ratio - 1)^3), nu = 2 on accept, mu *= nu, nu *= 2 on reject.
//
// One CTA per agent; vectors are K*N 2x2 complex blocks; every reduction has a fixed order.
#include <math.h>

#include "calib_internal.cuh"

namespace calib {
namespace {

constexpr int LM_THREADS = 256;

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
        const Blk p = load_blk(a.part + ((size_t)agent * a.n_chunks + ch) * KN * 8, blk);
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

// Sum of NV values over the CTA (float64, fixed order); results in out[0..NV).
template <int NV>
__device__ void block_sum_vec(double (&v)[NV], double* red, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
    __syncthreads();
    if (lane == 0)
        for (int i = 0; i < NV; ++i) red[w * NV + i] = v[i];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += red[j * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Remove the component of a data gradient G_k along the gauge orbit {J_k A : A anti-Hermitian}.
// g is invariant under J_k -> J_k U (C = c I_2, Eq. coh), so its exact gradient has none: the
// anti-Hermitian part of J_k^H G_k vanishes. Float32 residuals leave round-off there, which would
// otherwise steer the weakly determined gauge mode (curved only by the rho/2 penalty). With
// S = J^H J, solve (S A + A S)/2 = skew(J^H G) for A = [[i a, b + i c], [-b + i c, i d]] and set
// G <- G - J A (the h-orthogonal projection). Exact arithmetic leaves G unchanged.
__device__ void project_out_gauge(const float* J, float* G, int N, int K, double* red, double* sh) {
    for (int k = 0; k < K; ++k) {
        const float* Jk = J + (size_t)k * N * 8;
        float* Gk = G + (size_t)k * N * 8;
        double v[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            const float* j = Jk + p * 8;
            const float* g = Gk + p * 8;
            // S += J^H J (s0, s1, re s01, im s01); M += J^H G (4 complex, row-major)
            for (int m = 0; m < 2; ++m) {
                const double j0r = j[m * 4 + 0], j0i = j[m * 4 + 1], j1r = j[m * 4 + 2], j1i = j[m * 4 + 3];
                v[0] += j0r * j0r + j0i * j0i;
                v[1] += j1r * j1r + j1i * j1i;
                v[2] += j0r * j1r + j0i * j1i;
                v[3] += j0r * j1i - j0i * j1r;
                for (int c = 0; c < 2; ++c) {
                    const double gr = g[m * 4 + 2 * c], gi = g[m * 4 + 2 * c + 1];
                    // M[0][c] += conj(J[m][0]) G[m][c]; M[1][c] += conj(J[m][1]) G[m][c]
                    v[4 + 2 * c] += j0r * gr + j0i * gi;
                    v[5 + 2 * c] += j0r * gi - j0i * gr;
                    v[8 + 2 * c] += j1r * gr + j1i * gi;
                    v[9 + 2 * c] += j1r * gi - j1i * gr;
                }
            }
        }
        block_sum_vec<12>(v, red, sh);
        if (threadIdx.x == 0) {
            const double s0 = sh[0], s1 = sh[1], u = sh[2], w = sh[3];
            // skew(M): t0 = Im M00, t1 = Im M11, t2 + i t3 = (M01 - conj(M10)) / 2
            const double t0 = sh[5], t1 = sh[11];
            const double t2 = 0.5 * (sh[6] - sh[8]), t3 = 0.5 * (sh[7] + sh[9]);
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
            sh[12] = ok ? Mx[0][4] / Mx[0][0] : 0.0;  // a
            sh[13] = ok ? Mx[1][4] / Mx[1][1] : 0.0;  // d
            sh[14] = ok ? Mx[2][4] / Mx[2][2] : 0.0;  // b
            sh[15] = ok ? Mx[3][4] / Mx[3][3] : 0.0;  // c
        }
        __syncthreads();
        const float a = (float)sh[12], d = (float)sh[13], b = (float)sh[14], c = (float)sh[15];
        // A = [[i a, b + i c], [-b + i c, i d]]
        const float A00r = 0.f, A00i = a, A01r = b, A01i = c, A10r = -b, A10i = c, A11r = 0.f, A11i = d;
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            const float* j = Jk + p * 8;
            float* g = Gk + p * 8;
            for (int r = 0; r < 2; ++r) {
                const float jr0 = j[r * 4 + 0], ji0 = j[r * 4 + 1], jr1 = j[r * 4 + 2], ji1 = j[r * 4 + 3];
                // (J A)[r][0] = J[r][0] A00 + J[r][1] A10 ; (J A)[r][1] = J[r][0] A01 + J[r][1] A11
                g[r * 4 + 0] -= jr0 * A00r - ji0 * A00i + jr1 * A10r - ji1 * A10i;
                g[r * 4 + 1] -= jr0 * A00i + ji0 * A00r + jr1 * A10i + ji1 * A10r;
                g[r * 4 + 2] -= jr0 * A01r - ji0 * A01i + jr1 * A11r - ji1 * A11i;
                g[r * 4 + 3] -= jr0 * A01i + ji0 * A01r + jr1 * A11i + ji1 * A11r;
            }
        }
        __syncthreads();
    }
}

// Jacobi blocks G_pk = sum over slots incident on p of s_bk J_ok^H J_ok at the current J, via the
// circulant-diagonal slot table (two phases per diagonal, as in the sweeps).
__device__ void gram_blocks(const LMArgs& a, int agent, const float* J, float* Gout, float* Xs, float* Gs) {
    const int N = a.N, K = a.K, KN = K * N;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const Blk j = load_blk(J, blk);
        // X = J^H J: x00 = |J00|^2 + |J10|^2, x11 = |J01|^2 + |J11|^2, x01 = conj(J00) J01 + conj(J10) J11
        const float j00r = j.v[0], j00i = j.v[1], j01r = j.v[2], j01i = j.v[3];
        const float j10r = j.v[4], j10i = j.v[5], j11r = j.v[6], j11i = j.v[7];
        Xs[blk * 4 + 0] = j00r * j00r + j00i * j00i + j10r * j10r + j10i * j10i;
        Xs[blk * 4 + 1] = j01r * j01r + j01i * j01i + j11r * j11r + j11i * j11i;
        Xs[blk * 4 + 2] = j00r * j01r + j00i * j01i + j10r * j11r + j10i * j11i;
        Xs[blk * 4 + 3] = j00r * j01i - j00i * j01r + j10r * j11i - j10i * j11r;
        Gs[blk * 4 + 0] = Gs[blk * 4 + 1] = Gs[blk * 4 + 2] = Gs[blk * 4 + 3] = 0.f;
    }
    __syncthreads();
    const DiagDesc* dsc_agent = a.desc + (size_t)agent * a.D;
    for (int d = 0; d < a.D; ++d) {
        const DiagDesc dsc = dsc_agent[d];
        for (int phase = 0; phase < 2; ++phase) {
            for (int it = threadIdx.x; it < dsc.n * K; it += blockDim.x) {
                const int g = it / K, k = it - g * K;
                const int sl = a.slot[dsc.slot_off + g];
                const int f = sl & 0xff, s2 = (sl >> 8) & 0xff;
                const float w = a.spow[((size_t)dsc.slot_off + g) * K + k];
                const int dst = phase == 0 ? f : s2, src = phase == 0 ? s2 : f;
                float* G = Gs + (k * N + dst) * 4;
                const float* X = Xs + (k * N + src) * 4;
                G[0] += w * X[0]; G[1] += w * X[1]; G[2] += w * X[2]; G[3] += w * X[3];
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < KN * 4; i += blockDim.x) Gout[i] = Gs[i];
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

__global__ void __launch_bounds__(LM_THREADS) k_lm_eval(const LMArgs a, int mode) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[33];
    const int agent = blockIdx.x;
    const int N = a.N, K = a.K, KN = K * N;
    const size_t off = (size_t)agent * KN * 8;
    float* Xs = sm;
    float* Gs = sm + KN * 4;
    AgentState& st = a.st[agent];

    __shared__ double redv[32 * 12];
    __shared__ double shv[16];
    if (mode == LM_BEGIN_FROM_PARTIALS) {
        for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) store_blk(a.gradg + off, blk, sum_parts(a, agent, blk, KN));
        __syncthreads();
        project_out_gauge(a.J + off, a.gradg + off, N, K, redv, shv);
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
                g_t += a.part_cost[(size_t)agent * a.n_chunks + ch];
                dg += a.part_dcost[(size_t)agent * a.n_chunks + ch];
            }
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
            project_out_gauge(a.J + off, a.gradg + off, N, K, redv, shv);
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

__global__ void __launch_bounds__(LM_THREADS) k_cg_step(const LMArgs a) {
    __shared__ double red[33];
    const int agent = blockIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    AgentState& st = a.st[agent];
    const int stop = st.cg_stop;
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
__global__ void __launch_bounds__(LM_THREADS) k_lm_trial(const LMArgs a) {
    __shared__ double red[33];
    const int agent = blockIdx.x;
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

// calib_eval: L, g and grad L at a given J (sweep already ran on J), without touching the state.
__global__ void __launch_bounds__(LM_THREADS) k_eval_output(const LMArgs a, float* grad_out, double* L_out, double* g_out) {
    __shared__ double red[33];
    const int agent = blockIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const double rk = a.rho[blk / N];
        const Blk gg = sum_parts(a, agent, blk, KN);
        const Blk y = load_blk(a.Y + off, blk), j = load_blk(a.Jt + off, blk), bz = load_blk(a.BZ + off, blk);
        Blk gr;
#pragma unroll
        for (int i = 0; i < 8; ++i)
            gr.v[i] = (float)((double)gg.v[i] + 0.5 * (double)y.v[i] + 0.5 * rk * ((double)j.v[i] - (double)bz.v[i]));
        store_blk(grad_out + off, blk, gr);
    }
    const double pen = block_sum(penalty_part(a.Jt + off, a.Y + off, a.BZ + off, a.rho, N, KN), red);
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (int ch = 0; ch < a.n_chunks; ++ch) g += a.part_cost[(size_t)agent * a.n_chunks + ch];
        if (g_out) g_out[agent] = g;
        if (L_out) L_out[agent] = g + pen;
    }
}

// calib_hessvec: out = H_GN eta + rho/2 eta (eta passed in a.p).
__global__ void __launch_bounds__(LM_THREADS) k_hv_output(const LMArgs a, float* out) {
    const int agent = blockIdx.x;
    const int N = a.N, KN = a.K * N;
    const size_t off = (size_t)agent * KN * 8;
    for (int blk = threadIdx.x; blk < KN; blk += blockDim.x) {
        const float h = 0.5f * a.rho[blk / N];
        const Blk hp = sum_parts(a, agent, blk, KN);
        const Blk e = load_blk(a.p + off, blk);
        Blk o;
#pragma unroll
        for (int i = 0; i < 8; ++i) o.v[i] = hp.v[i] + h * e.v[i];
        store_blk(out + off, blk, o);
    }
}

}  // namespace

cudaError_t prepare_lm_kernels() {
    return cudaFuncSetAttribute(k_lm_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}

cudaError_t launch_lm_eval(const LMArgs& a, int mode, cudaStream_t s) {
    const size_t smem = (size_t)a.K * a.N * 4 * sizeof(float) * 2;
    k_lm_eval<<<a.A, LM_THREADS, smem, s>>>(a, mode);
    return cudaGetLastError();
}
cudaError_t launch_cg_step(const LMArgs& a, cudaStream_t s) {
    k_cg_step<<<a.A, LM_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_lm_trial(const LMArgs& a, cudaStream_t s) {
    k_lm_trial<<<a.A, LM_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_eval_output(const LMArgs& a, float* grad_out, double* L_out, double* g_out, cudaStream_t s) {
    k_eval_output<<<a.A, LM_THREADS, 0, s>>>(a, grad_out, L_out, g_out);
    return cudaGetLastError();
}
cudaError_t launch_hv_output(const LMArgs& a, float* out, cudaStream_t s) {
    k_hv_output<<<a.A, LM_THREADS, 0, s>>>(a, out);
    return cudaGetLastError();
}

}  // namespace calib
