// Fusion-centre and dual steps of C-ADMM (Section 3): first-iteration gauge projection,
// the closed-form Z-update (Eq. Zest), the dual update (Eq. M3) and the per-iteration
// residuals of Section 4. On one GPU the paper's agent -> fusion centre -> agent messages
// become a device reduction over the P agents of each solution interval, ordered by the stream.
#include <math.h>

#include "calib_internal.cuh"
#include "df.cuh"

namespace calib {
namespace {

constexpr int CT = 256;

__device__ double bsum(double v, double* red) {
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

struct C2 { double r, i; };
__device__ __forceinline__ C2 cm(C2 a, C2 b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ C2 cconj(C2 a) { return {a.r, -a.i}; }
__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return {a.r + b.r, a.i + b.i}; }

// First C-ADMM iteration (Section 3, initialisation): rotate each agent's J_k by the unitary
// polar factor U of M = J_k^H J_ref,k (the 2x2 Procrustes solution, min_U ||J_ref - J U||), the
// reference being the middle agent (index P_g / 2) of the same consensus problem. For 2x2 M with
// det M = |det M| e^{i theta}: U = (M + e^{i theta} adj(M)^H) / sqrt(||M||_F^2 + 2 |det M|).
// The stored data gradient and Jacobi blocks are rotated with J (grad g(JU) = grad g(J) U,
// G(JU) = U^H G U) since g is invariant under the common unitary.
// One warp per direction: M accumulated over the stations in float32 and reduced across the warp,
// U formed from it in float64 by lane 0 and broadcast, and J, the gradient and G rotated in float32
// (they are float32 data).
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
struct F2 { float r, i; };
__device__ __forceinline__ F2 fm(F2 a, F2 b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ F2 fcm(F2 a, F2 b) { return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r}; }  // conj(a) b
__device__ __forceinline__ F2 fadd(F2 a, F2 b) { return {a.r + b.r, a.i + b.i}; }

__global__ void __launch_bounds__(CT) k_gauge(const ConsArgs a) {
    const int agent = blockIdx.x;
    const int iv = agent / a.P, f = agent - iv * a.P;
    const int g = f % a.G, Pg = a.P / a.G;
    const int ref = iv * a.P + g + a.G * (Pg / 2);
    if (agent == ref) return;
    const int N = a.N, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < a.K; k += nw) {
        const float* Ja = a.J + ((size_t)agent * a.K + k) * N * 8;
        const float* Jr = a.J + ((size_t)ref * a.K + k) * N * 8;
        float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // M[i][j] at 2 (2 i + j) (re, im)
        for (int p = lane; p < N; p += 32) {
            F2 ja[4], jr[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ja[e] = {Ja[p * 8 + 2 * e], Ja[p * 8 + 2 * e + 1]};
                jr[e] = {Jr[p * 8 + 2 * e], Jr[p * 8 + 2 * e + 1]};
            }
            // M[i][j] += sum_m conj(Ja[m][i]) Jr[m][j]
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const F2 t = fadd(fcm(ja[0 * 2 + i], jr[0 * 2 + j]), fcm(ja[1 * 2 + i], jr[1 * 2 + j]));
                    m[2 * (2 * i + j)] += t.r;
                    m[2 * (2 * i + j) + 1] += t.i;
                }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) m[e] = warp_sum_f32(m[e]);
        float u[8];
        if (lane == 0) {
            const C2 M00 = {m[0], m[1]}, M01 = {m[2], m[3]}, M10 = {m[4], m[5]}, M11 = {m[6], m[7]};
            const C2 det = cadd(cm(M00, M11), {-(cm(M01, M10).r), -(cm(M01, M10).i)});
            const double adet = hypot(det.r, det.i);
            const C2 ph = adet > 0 ? C2{det.r / adet, det.i / adet} : C2{1.0, 0.0};
            // adj(M) = [[M11, -M01], [-M10, M00]]; adj(M)^H = [[conj M11, -conj M10], [-conj M01, conj M00]]
            const C2 A00 = cconj(M11), A01 = {-M10.r, M10.i}, A10 = {-M01.r, M01.i}, A11 = cconj(M00);
            const double fro = M00.r * M00.r + M00.i * M00.i + M01.r * M01.r + M01.i * M01.i +
                               M10.r * M10.r + M10.i * M10.i + M11.r * M11.r + M11.i * M11.i;
            const double sq = sqrt(fro + 2.0 * adet);
            C2 U[4] = {{1, 0}, {0, 0}, {0, 0}, {1, 0}};
            if (sq > 0) {
                const double is = 1.0 / sq;
                const C2 u00 = cadd(M00, cm(ph, A00)), u01 = cadd(M01, cm(ph, A01));
                const C2 u10 = cadd(M10, cm(ph, A10)), u11 = cadd(M11, cm(ph, A11));
                U[0] = {u00.r * is, u00.i * is};
                U[1] = {u01.r * is, u01.i * is};
                U[2] = {u10.r * is, u10.i * is};
                U[3] = {u11.r * is, u11.i * is};
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                u[2 * e] = (float)U[e].r;
                u[2 * e + 1] = (float)U[e].i;
            }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = __shfl_sync(0xffffffffu, u[e], 0);
        const F2 U[4] = {{u[0], u[1]}, {u[2], u[3]}, {u[4], u[5]}, {u[6], u[7]}};
        float* Jw = a.J + ((size_t)agent * a.K + k) * N * 8;
        float* Gw = a.gradg + ((size_t)agent * a.K + k) * N * 8;
        float* Hw = a.Gm + ((size_t)agent * a.K + k) * N * 4;
        for (int p = lane; p < N; p += 32) {
#pragma unroll
            for (int which = 0; which < 2; ++which) {
                float* X = (which == 0 ? Jw : Gw) + p * 8;
                F2 x[4], y[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) x[e] = {X[2 * e], X[2 * e + 1]};
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int n = 0; n < 2; ++n) y[r * 2 + n] = fadd(fm(x[r * 2 + 0], U[0 * 2 + n]), fm(x[r * 2 + 1], U[1 * 2 + n]));
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    X[2 * e] = y[e].r;
                    X[2 * e + 1] = y[e].i;
                }
            }
            // G <- U^H G U
            float* Gp = Hw + p * 4;
            const F2 Gm_[4] = {{Gp[0], 0.f}, {Gp[2], Gp[3]}, {Gp[2], -Gp[3]}, {Gp[1], 0.f}};
            F2 T[4], R[4];
#pragma unroll
            for (int r = 0; r < 2; ++r)  // T = G U
#pragma unroll
                for (int n = 0; n < 2; ++n) T[r * 2 + n] = fadd(fm(Gm_[r * 2 + 0], U[0 * 2 + n]), fm(Gm_[r * 2 + 1], U[1 * 2 + n]));
#pragma unroll
            for (int r = 0; r < 2; ++r)  // R = U^H T
#pragma unroll
                for (int n = 0; n < 2; ++n) R[r * 2 + n] = fadd(fcm(U[0 * 2 + r], T[0 * 2 + n]), fcm(U[1 * 2 + r], T[1 * 2 + n]));
            Gp[0] = R[0].r;
            Gp[1] = R[3].r;
            Gp[2] = R[1].r;
            Gp[3] = R[1].i;
        }
    }
}

// One C-ADMM fusion-centre and dual step for one (consensus problem, direction) and ZJ consecutive
// (station, entry) positions, in double-float arithmetic (df.cuh; the GPU's float64 rate is far
// below its float32 rate and this step has few bytes per operation):
//   Z-update (Eq. Zest in the reshaped form z = vec(R P^T) of Section 3):
//     Z_k = (1/rho_k) Pinv sum_f b(f) (Y_fk + rho_k J_fk); the ZG warps split the problem's agents
//     (warp w takes the agents w, w + ZG, ...) and their sums are added in warp order (a fixed
//     order: results do not depend on timing); Z, Zprev are stored in float64, and this CTA's share
//     of ||Z_k^{n+1} - Z_k^n||^2 (the dual residual, Section 4) goes to its own slot of dual2;
//   Y-update (Eq. M3) of every agent f of the problem at the same positions, from the new Z held in
//     shared memory: B_f Z = sum_l b_l(f) Z_l, D = J_f - B_f Z, Y_f += rho_k D (rounded once to
//     float32), and the agent's shares of ||D||^2 and of Re tr(Y^H D) + rho/2 ||D||^2 (Eq. sumtrace2,
//     with the new Y) over these positions, in float32, summed by k_records.
constexpr int ZJ = 32;  // (station, entry) positions per CTA: one per lane
constexpr int ZG = 4;   // warps per CTA, each over every ZG-th agent of the problem

// MB: the basis size rounded up to a compiled bucket (every loop over the basis is unrolled to MB).
template <int MB>
__global__ void __launch_bounds__(ZJ * ZG) k_zy_update(const ConsArgs a) {
    __shared__ float2 Rs[ZG][MB][ZJ];
    __shared__ float2 Zs[MB][ZJ];
    __shared__ double red[33];
    const int ivk = blockIdx.x;  // (consensus problem, direction)
    const int k = ivk % a.K, pb = ivk / a.K;
    const int iv = pb / a.G, g = pb - iv * a.G, Pg = a.P / a.G;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int j = blockIdx.y * ZJ + lane;  // (station, entry) = (j / 8, j % 8)
    const int NE = a.N * 8, M = a.M;
    const bool on = j < NE;
    const float rk = a.rho[k];
    const size_t stride = (size_t)a.G * a.K * NE;  // next agent of the problem, same direction
    const size_t o0 = (((size_t)iv * a.P + g) * a.K + k) * NE + j;
    DF R[MB];
#pragma unroll
    for (int l = 0; l < MB; ++l) R[l] = DF{0.f, 0.f};
    if (on) {
#pragma unroll 2
        for (int jj = grp; jj < Pg; jj += ZG) {
            const size_t o = o0 + (size_t)jj * stride;
            const DF v = df_add(df_prod(rk, __ldg(a.J + o)), DF{__ldg(a.Y + o), 0.f});  // Y + rho J
            const float2* bf = a.basis_df + (size_t)(g + a.G * jj) * M;
#pragma unroll
            for (int l = 0; l < MB; ++l)
                if (l < M) R[l] = df_fma(df_load(bf + l), v, R[l]);
        }
    }
#pragma unroll
    for (int l = 0; l < MB; ++l)
        if (l < M) Rs[grp][l][lane] = make_float2(R[l].hi, R[l].lo);
    __syncthreads();
    // the warps' sums added in warp order (R_m identical in every warp); warp w forms the Z_l with
    // l = w mod ZG
    double dz2 = 0.0;
    if (on) {
#pragma unroll
        for (int m = 0; m < MB; ++m) {
            if (m >= M) continue;
            R[m] = df_load(&Rs[0][m][lane]);
#pragma unroll
            for (int w = 1; w < ZG; ++w) R[m] = df_add(R[m], df_load(&Rs[w][m][lane]));
        }
        const float2* Pinv = a.Pinv_df + (size_t)g * M * M;
        const DF ri = df_load(a.rinv_df + k);
        for (int l = grp; l < M; l += ZG) {
            DF z{0.f, 0.f};
#pragma unroll
            for (int m = 0; m < MB; ++m)
                if (m < M) z = df_fma(df_load(Pinv + l * M + m), R[m], z);
            z = df_mul(z, ri);
            const size_t zo = (((size_t)pb * a.K + k) * M + l) * NE + j;
            const double zd = df_to_double(z), old = a.Z[zo];
            a.Zprev[zo] = old;
            a.Z[zo] = zd;
            dz2 = fma(zd - old, zd - old, dz2);
            Zs[l][lane] = make_float2(z.hi, z.lo);
        }
    }
    dz2 = bsum(dz2, red);  // its barriers also publish Zs
    if (threadIdx.x == 0) a.dual2[(size_t)ivk * Z_SLOTS + blockIdx.y] = dz2;

    DF zl[MB];
#pragma unroll
    for (int l = 0; l < MB; ++l) zl[l] = (on && l < M) ? df_load(&Zs[l][lane]) : DF{0.f, 0.f};
    for (int jj = grp; jj < Pg; jj += ZG) {  // the same trip count in every lane of the warp
        const int f = g + a.G * jj;
        float dd = 0.f, pen = 0.f;
        if (on) {
            const size_t o = o0 + (size_t)jj * stride;
            const float2* bf = a.basis_df + (size_t)f * M;
            DF bz{0.f, 0.f};
#pragma unroll
            for (int l = 0; l < MB; ++l)
                if (l < M) bz = df_fma(df_load(bf + l), zl[l], bz);
            const float y = a.Y[o];
            const DF d = df_add(DF{a.J[o], 0.f}, df_neg(bz));  // J - B Z
            DF t = df_prod(rk, d.hi);
            t.lo = __fmaf_rn(rk, d.lo, t.lo);
            const float ynew = df_add(t, DF{y, 0.f}).hi;  // Y + rho D
            a.Y[o] = ynew;
            a.BZ[o] = bz.hi;
            dd = d.hi * d.hi;
            pen = fmaf(ynew, d.hi, 0.5f * rk * dd);
        }
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) {
            dd += __shfl_xor_sync(0xffffffffu, dd, w);
            pen += __shfl_xor_sync(0xffffffffu, pen, w);
        }
        if (lane == 0) {
            const size_t po = (((size_t)iv * a.P + f) * a.K + k) * Z_SLOTS + blockIdx.y;
            a.prim_part[po] = dd;
            a.pen_part[po] = pen;
        }
    }
}

// BZ_i = sum_l b_l(f_i) Z_l for a Z set from outside the iteration (calib_set_consensus), with
// the per-agent ||J_ik - BZ_ik|| and L_i(J_i, Z, Y_i) = g_i + Re tr(Y^H D) + rho/2 ||D||^2
// (Eq. sumtrace2); Y is left as it is. One CTA per agent, one thread per real entry of a
// (direction, station) block (independent loads); a block's 8 entries sit in 8 aligned lanes and
// are summed by shuffles, the per-direction norms over the stations by one warp each (fixed order).
__global__ void __launch_bounds__(CT) k_bz(const ConsArgs a) {
    __shared__ double red[33];
    extern __shared__ double dds[];  // [K][N] ||J - BZ||^2 per block
    const int agent = blockIdx.x;
    const int iv = agent / a.P, f = agent - iv * a.P;
    const int pb = iv * a.G + f % a.G;  // the agent's consensus problem
    const int N = a.N, KN8 = a.K * N * 8, M = a.M;
    double bl[MAX_M];
#pragma unroll
    for (int l = 0; l < MAX_M; ++l) bl[l] = l < M ? a.basis[f * M + l] : 0.0;
    // B Z and the difference J - B Z in float64; the squares and the penalty terms of that
    // difference (records only) in float32, summed in float64 across the CTA.
    float pen = 0.f;
    const int KN8r = (KN8 + blockDim.x - 1) / blockDim.x * blockDim.x;  // every lane runs every trip
    for (int i = threadIdx.x; i < KN8r; i += blockDim.x) {
        const bool on = i < KN8;  // KN8 is a multiple of 8: a block's 8 lanes are all on or all off
        float dd = 0.f;
        if (on) {
            const int k = i / (N * 8), pe = i - k * N * 8;  // pe = station * 8 + entry
            const size_t o = (size_t)agent * KN8 + i;
            const double* z = a.Z + ((size_t)pb * a.K + k) * M * N * 8 + pe;  // Z[pb][k][l][p][e] at l = 0
            double bz = 0.0;
#pragma unroll
            for (int l = 0; l < MAX_M; ++l)
                if (l < M) bz = fma(bl[l], z[(size_t)l * N * 8], bz);
            const double d = (double)a.J[o] - bz;
            const float ynew = a.Y[o];
            a.BZ[o] = (float)bz;
            const float df = (float)d, rf = a.rho[k];
            dd = df * df;
            pen += fmaf(ynew, df, 0.5f * rf * dd);
        }
        for (int w = 4; w > 0; w >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, w);
        if (on && (i & 7) == 0) dds[i >> 3] = (double)dd;
    }
    const double pen_d = bsum((double)pen, red);  // its barriers also publish dds
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k < a.K; k += nw) {
        double s = 0.0;
        for (int p = lane; p < N; p += 32) s += dds[k * N + p];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && a.prim) a.prim[(size_t)agent * a.K + k] = sqrt(s);
    }
    if (threadIdx.x == 0) a.st[agent].L = a.st[agent].g + pen_d;
}

// Per-iteration record (Section 4): primal, dual, objective, data residual norm, and each agent's
// L_i = g_i + Re tr(Y^H D) + rho/2 ||D||^2 (Eq. sumtrace2) from the shares k_zy_update wrote. One
// warp per agent, REC_AGENTS agents per CTA, every sum in a fixed order; each CTA writes its sums
// to its own slot, and the CTA that finishes last (counted with an atomic after a fence; no CTA
// waits) adds the slots in CTA order, writes the record and resets the count.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(REC_AGENTS * 32) k_records(const ConsArgs a) {
    __shared__ double sp[REC_AGENTS][3];
    __shared__ double red[33];
    __shared__ int last_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int agent = blockIdx.x * REC_AGENTS + w;
    const int zs = (a.N * 8 + ZJ - 1) / ZJ;  // Z-update CTAs per (consensus problem, direction)
    double prim = 0.0, obj = 0.0, g = 0.0;
    if (agent < a.A) {
        // the float32 shares are summed in float32 (the records' precision); the agents in float64
        // lane y holds chunk y (zs <= 32) of every direction: all loads are issued together
        float s[MAX_K], q[MAX_K];
#pragma unroll
        for (int k = 0; k < MAX_K; ++k) {
            s[k] = q[k] = 0.f;
            if (k < a.K && lane < zs) {
                const size_t i = ((size_t)agent * a.K + k) * Z_SLOTS + lane;
                s[k] = a.prim_part[i];
                q[k] = a.pen_part[i];
            }
        }
        g = a.st[agent].g;
        float pen = 0.f;
#pragma unroll
        for (int k = 0; k < MAX_K; ++k) {
            if (k >= a.K) continue;
            prim += (double)sqrtf(warp_sum_f(s[k]));  // ||J_ik - B_i Z_k||
            pen += warp_sum_f(q[k]);
        }
        obj = g + (double)pen;
        if (lane == 0) a.st[agent].L = obj;
    }
    if (lane == 0) {
        sp[w][0] = prim;
        sp[w][1] = obj;
        sp[w][2] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < REC_AGENTS; ++i)
            for (int c = 0; c < 3; ++c) t[c] += sp[i][c];
        for (int c = 0; c < 3; ++c) a.rec_part[(size_t)blockIdx.x * 3 + c] = t[c];
        __threadfence();
        last_s = atomicAdd(a.rec_count, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    double pr = 0.0, dual = 0.0, ob = 0.0, gg = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        pr += __ldcg(a.rec_part + (size_t)i * 3 + 0);
        ob += __ldcg(a.rec_part + (size_t)i * 3 + 1);
        gg += __ldcg(a.rec_part + (size_t)i * 3 + 2);
    }
    for (int i = threadIdx.x; i < a.I * a.G * a.K; i += blockDim.x) {
        double d2 = 0.0;
        for (int y = 0; y < zs; ++y) d2 += a.dual2[(size_t)i * Z_SLOTS + y];
        dual += sqrt(d2);
    }
    pr = bsum(pr, red);
    dual = bsum(dual, red);
    ob = bsum(ob, red);
    gg = bsum(gg, red);
    if (threadIdx.x == 0) {
        const int it = *a.iter_counter;
        if (it < a.max_iters) {
            double* o = a.stats + (size_t)it * 4;
            o[0] = pr / sqrt(4.0 * a.N) / ((double)a.A * a.K);
            o[1] = dual / sqrt(4.0 * a.M * a.N) / ((double)a.I * a.G * a.K);
            o[2] = ob;
            o[3] = sqrt(gg);
        }
        *a.iter_counter = it + 1;
        *a.rec_count = 0;
    }
}

__global__ void k_identity(float* J, long long n_blocks) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_blocks) return;
    float4* p = reinterpret_cast<float4*>(J + i * 8);
    p[0] = make_float4(1.f, 0.f, 0.f, 0.f);
    p[1] = make_float4(0.f, 0.f, 1.f, 0.f);
}

}  // namespace

cudaError_t launch_gauge(const ConsArgs& a, cudaStream_t s) {
    k_gauge<<<a.A, CT, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_zy_update(const ConsArgs& a, cudaStream_t s) {
    const int zs = (a.N * 8 + ZJ - 1) / ZJ;
    if (zs > Z_SLOTS || a.M > MAX_M) return cudaErrorInvalidConfiguration;
    const dim3 grid(a.I * a.G * a.K, zs);
    if (a.M <= 2)
        k_zy_update<2><<<grid, ZJ * ZG, 0, s>>>(a);
    else if (a.M <= 4)
        k_zy_update<4><<<grid, ZJ * ZG, 0, s>>>(a);
    else if (a.M <= 8)
        k_zy_update<8><<<grid, ZJ * ZG, 0, s>>>(a);
    else
        k_zy_update<MAX_M><<<grid, ZJ * ZG, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bz_only(const ConsArgs& a, cudaStream_t s) {
    k_bz<<<a.A, CT, (size_t)a.K * a.N * sizeof(double), s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_records(const ConsArgs& a, cudaStream_t s) {
    k_records<<<(a.A + REC_AGENTS - 1) / REC_AGENTS, REC_AGENTS * 32, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_identity(float* J, long long n_blocks, cudaStream_t s) {
    k_identity<<<(unsigned)((n_blocks + 255) / 256), 256, 0, s>>>(J, n_blocks);
    return cudaGetLastError();
}

}  // namespace calib
