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
#include "lm_device.cuh"

namespace calib {
namespace {

constexpr int LM_THREADS = 256;

__global__ void __launch_bounds__(LM_THREADS) k_lm_eval(const LMArgs a, int mode) {
    extern __shared__ __align__(16) float sm[];
    __shared__ double red[33];
    lm_eval_dev(a, blockIdx.x, mode, sm, red);
}

__global__ void __launch_bounds__(LM_THREADS) k_cg_step(const LMArgs a) {
    __shared__ double red[33];
    cg_step_dev(a, blockIdx.x, red);
}

__global__ void __launch_bounds__(LM_THREADS) k_lm_trial(const LMArgs a) {
    __shared__ double red[33];
    lm_trial_dev(a, blockIdx.x, red);
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
