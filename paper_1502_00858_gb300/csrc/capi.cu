// C ABI of libcalib.so (declared in include/calib.h): context, device layout, the C-ADMM
// iteration schedule (Section 3, steps D1-D3) captured into CUDA graphs, and the data paths.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "calib.h"
#include "calib_internal.cuh"
#include "df.cuh"
#include "tma.cuh"

namespace calib {

// One CTA waits, with the same bounded wait as the sweeps' copy ring, on an mbarrier phase that
// completes only if complete_phase is set (one arrival on a count-1 barrier). No copy is issued, so
// when the wait gives up nothing is in flight and the CTA can return at once.
__global__ void k_wait_selftest(int complete_phase, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (complete_phase && threadIdx.x == 0) mbar_arrive(&bar);
    const bool ok = mbar_wait_bounded(&bar, 0u);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, STATUS_TIMEOUT);
}

}  // namespace calib

using namespace calib;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(expr)                                                                                \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess) return fail(CALIB_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

struct ProfPair {
    cudaEvent_t a, b;
    int kind;  // 0 residual or trial sweep, 1 Hessian sweep, 2 statistics Hessian, 3 statistics trial
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    std::vector<ProfPair> prof;
};

}  // namespace

struct TuneEntry {
    int v;          // candidate split
    double hv, tr;  // ms: n_cg Hessian passes with their PCG steps; the trial pass with its reduction
};

struct calib_ctx {
    int dev = 0;
    int N = 0, B = 0, K = 0, P = 0, M = 0, I = 0, A = 0, D = 0;
    int G = 1;  // frequency groups per interval: I * G consensus problems of P / G agents
    int n_lm = 10, n_cg = 4, chunk_diags = 1, n_chunks = 1, slots_max = 4;
    int jupdate = 0;               // CALIB_JUPDATE_LM, CALIB_JUPDATE_RTR or CALIB_JUPDATE_SAGE
    int n_sage = 1;                // SAGE sweeps over the directions per J-update
    bool tune_pending = false;     // work split chosen by the autotuner at the first iteration
    // statistics sweeps: grid = sms * m CTAs (at most A*D), balanced contiguous item ranges; the
    // Hessian and trial passes are split independently
    int sms = 1;
    struct Partition {
        int m = 4, grid = 1, stride = 1;
        int* pn = nullptr;         // [A] pieces (CTAs) meeting each agent
    } part_hv, part_tr;
    std::vector<TuneEntry> tune_log;  // per candidate split: ms of the Hessian half and of the trial half
    int TT_res = 1, TT_hv = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    std::vector<int32_t> pq;
    std::vector<double> freqs, basis, rho, Pinv;
    std::vector<float> rho_f;
    std::vector<int> T;
    int Tmax = 1;  // largest samples per agent
    std::vector<long long> vis_off, coh_off;   // user layout offsets per agent (float2 units)
    long long user_v = 0, user_c = 0;           // user layout totals (float2)

    // layout (depends on flags)
    std::vector<DiagDesc> desc_h;
    std::vector<int> slot_h, slot_b_h;
    long long int_v = 0, int_c = 0;             // internal totals (float2)
    long long int_u = 0, int_s = 0;             // sufficient-statistics totals (float2)
    double alg_bytes[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // algorithmic bytes per launch of each profiled kind
    double alg_flops[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // algorithmic real flops per launch of each profiled kind
    std::vector<uint8_t> flags_h;

    // device
    float2 *V = nullptr, *C = nullptr, *ssU = nullptr, *ssS = nullptr;
    int formulation = 0;  // 0 sufficient statistics, 1 direct
    bool ss_dirty = true;
    DiagDesc* desc = nullptr;
    int *slot = nullptr, *slot_b = nullptr, *T_d = nullptr;
    int2* inc = nullptr;
    float* gw = nullptr;  // [A][K][N][N] Jacobi weights
    long long *vis_off_d = nullptr, *coh_off_d = nullptr;
    float *J = nullptr, *Jt = nullptr, *Y = nullptr, *BZ = nullptr, *gradg = nullptr, *grad = nullptr;
    float *x = nullptr, *r = nullptr, *p = nullptr, *Gm = nullptr;
    float *evJ = nullptr, *evE = nullptr, *evOut = nullptr;
    float* part = nullptr;
    double* part_cost = nullptr;
    double* part_dcost = nullptr;
    double *Z = nullptr, *Zprev = nullptr, *basis_d = nullptr, *Pinv_d = nullptr, *freqs_d = nullptr;
    float* rho_d = nullptr;
    AgentState* st = nullptr;
    double* prim = nullptr;
    double* dual2 = nullptr;
    float2 *basis_df = nullptr, *Pinv_df = nullptr, *rinv_df = nullptr;  // double-float tables
    float *prim_part = nullptr, *pen_part = nullptr;  // per-CTA shares of the fused Z/Y update
    double* rec_part = nullptr;                       // per-CTA sums of the record kernel
    int* rec_count = nullptr;
    double* stats = nullptr;
    int max_iters = 0;
    int* iter_counter = nullptr;
    int* status = nullptr;
    double* evL = nullptr;
    double* evG = nullptr;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    // SAGE: one direction's one-direction problem (statistics and per-agent vectors, K = 1)
    float2 *sgU = nullptr, *sgS = nullptr;
    float *sgJ = nullptr, *sgJt = nullptr, *sgY = nullptr, *sgBZ = nullptr, *sgGradg = nullptr, *sgGrad = nullptr;
    float *sgX = nullptr, *sgR = nullptr, *sgP = nullptr, *sgGm = nullptr;
    AgentState* sgSt = nullptr;
    float *ws_prev = nullptr, *ws_mlp = nullptr;   // warm start: previous J, network J
    double *ws_L = nullptr, *xf_d = nullptr;         // [2A] L at both starts; [A] normalised frequency
    int* ws_chose = nullptr;

    bool data_set = false, coh_set = false;
    bool cold = true, need_eval = true;
    long long iters_done = 0;  // C-ADMM iterations since the last cold start or warm state

    std::map<std::tuple<int, int, int, int>, GraphEntry> graphs;
    long long launches = 0;
    bool profiling = false;
    // 4 sweep kinds, the PCG step, the LM evaluation, the statistics pass, the fusion-centre step
    // (gauge, Z-update, Y-update and records of one iteration, timed together)
    static constexpr int PROF_KINDS = 8;
    double prof_ms[PROF_KINDS] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_n[PROF_KINDS] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

SweepArgs sweep_args(calib_ctx* c, int mode, const float* J, const float* eta) {
    const bool hv = mode == SWEEP_HESSVEC;
    SweepArgs a{};
    a.V = c->V;
    a.C = c->C;
    a.desc = c->desc;
    a.slot = c->slot;
    a.T = c->T_d;
    a.J = J;
    a.eta = eta;
    a.part = c->part;
    a.part_cost = c->part_cost;
    a.part_dcost = c->part_dcost;
    a.status = c->status;
    a.A = c->A;
    a.N = c->N;
    a.K = c->K;
    a.D = c->D;
    a.n_chunks = c->n_chunks;
    a.chunk_diags = c->chunk_diags;
    a.TT = hv ? c->TT_hv : c->TT_res;
    a.slots_max = c->slots_max;
    return a;
}

// ss_parts: the partials come from a statistics sweep (per-agent piece counts), else from a
// direct sweep (n_chunks per agent).
enum PartsFrom { PARTS_DIRECT, PARTS_SS_HESSIAN, PARTS_SS_TRIAL };

// Where the partials the LM kernel reduces come from: a direct sweep (n_chunks per agent) or a
// statistics sweep (per-agent piece counts of its partition).
LMArgs lm_args(calib_ctx* c, PartsFrom from) {
    LMArgs a{};
    a.part = c->part;
    a.part_cost = c->part_cost;
    a.part_dcost = c->part_dcost;
    const calib_ctx::Partition* pt = from == PARTS_SS_HESSIAN ? &c->part_hv : from == PARTS_SS_TRIAL ? &c->part_tr : nullptr;
    a.part_n = pt ? pt->pn : nullptr;
    a.part_stride = pt ? pt->stride : c->n_chunks;
    a.J = c->J;
    a.Jt = c->Jt;
    a.Y = c->Y;
    a.BZ = c->BZ;
    a.gradg = c->gradg;
    a.grad = c->grad;
    a.x = c->x;
    a.r = c->r;
    a.p = c->p;
    a.Gm = c->Gm;
    a.st = c->st;
    a.rho = c->rho_d;
    a.gw = c->gw;
    a.A = c->A;
    a.N = c->N;
    a.K = c->K;
    a.D = c->D;
    a.tau = 1e-3;
    a.cost_from_decrease = c->formulation == 0 ? 1 : 0;
    return a;
}

SSArgs ss_args(calib_ctx* c, const float* J, const float* eta, bool hessvec) {
    SSArgs a{};
    a.U = c->ssU;
    a.S = c->ssS;
    a.J = J;
    a.eta = eta;
    a.part = c->part;
    a.part_dcost = c->part_dcost;
    a.status = c->status;
    a.A = c->A;
    a.N = c->N;
    a.K = c->K;
    a.D = c->D;
    a.NP = (c->N + 3) / 4 * 4;
    a.part_stride = hessvec ? c->part_hv.stride : c->part_tr.stride;
    return a;
}

// The one-direction problem of direction k in the SAGE J-update: its statistics and vectors (K = 1).
SSArgs sage_ss_args(calib_ctx* c, bool hessvec) {
    SSArgs a = ss_args(c, c->sgJ, hessvec ? c->sgP : c->sgJt, hessvec);
    a.U = c->sgU;
    a.S = c->sgS;
    a.K = 1;
    return a;
}

LMArgs sage_lm_args(calib_ctx* c, PartsFrom from, int k) {
    LMArgs a = lm_args(c, from);
    a.J = c->sgJ;
    a.Jt = c->sgJt;
    a.Y = c->sgY;
    a.BZ = c->sgBZ;
    a.gradg = c->sgGradg;
    a.grad = c->sgGrad;
    a.x = c->sgX;
    a.r = c->sgR;
    a.p = c->sgP;
    a.Gm = c->sgGm;
    a.gw = nullptr;  // the trust-region kernels use no Jacobi blocks
    a.st = c->sgSt;
    a.rho = c->rho_d + k;
    a.K = 1;
    a.cost_from_decrease = 1;
    return a;
}

SageArgs sage_args(calib_ctx* c) {
    SageArgs g{};
    g.U = c->ssU;
    g.S = c->ssS;
    g.J = c->J;
    g.Y = c->Y;
    g.BZ = c->BZ;
    g.J_out = c->J;
    g.U1 = c->sgU;
    g.S1 = c->sgS;
    g.J1 = c->sgJ;
    g.Jt1 = c->sgJt;
    g.Y1 = c->sgY;
    g.BZ1 = c->sgBZ;
    g.A = c->A;
    g.D = c->D;
    g.NP = (c->N + 3) / 4 * 4;
    g.K = c->K;
    g.N = c->N;
    return g;
}

// Split the A*D items of the statistics sweeps over grid = min(A*D, sms * m) CTAs and record how
// many CTAs meet each agent (the pieces its reductions sum). CTA c takes items
// [floor(c W / G), floor((c+1) W / G)); item i lies in CTA ((i+1) G - 1) / W.
int set_partition(calib_ctx* c, calib_ctx::Partition& pt, int m) {
    const long long W = (long long)c->A * c->D;
    const long long G = std::max(1LL, std::min(W, (long long)c->sms * m));
    std::vector<int> pn(c->A);
    int stride = 1;
    for (int a = 0; a < c->A; ++a) {
        const long long c0 = (((long long)a * c->D + 1) * G - 1) / W;
        const long long c1 = (((long long)a * c->D + c->D) * G - 1) / W;
        pn[a] = (int)(c1 - c0 + 1);
        stride = std::max(stride, pn[a]);
    }
    CK(cudaMemcpy(pt.pn, pn.data(), pn.size() * sizeof(int), cudaMemcpyHostToDevice));
    pt.m = m;
    pt.grid = (int)G;
    pt.stride = stride;
    return CALIB_OK;
}

ConsArgs cons_args(calib_ctx* c) {
    ConsArgs a{};
    a.J = c->J;
    a.gradg = c->gradg;
    a.Gm = c->Gm;
    a.Y = c->Y;
    a.BZ = c->BZ;
    a.Z = c->Z;
    a.Zprev = c->Zprev;
    a.basis = c->basis_d;
    a.Pinv = c->Pinv_d;
    a.rho = c->rho_d;
    a.st = c->st;
    a.prim = c->prim;
    a.dual2 = c->dual2;
    a.basis_df = c->basis_df;
    a.Pinv_df = c->Pinv_df;
    a.rinv_df = c->rinv_df;
    a.prim_part = c->prim_part;
    a.pen_part = c->pen_part;
    a.rec_part = c->rec_part;
    a.rec_count = c->rec_count;
    a.stats = c->stats;
    a.iter_counter = c->iter_counter;
    a.A = c->A;
    a.I = c->I;
    a.P = c->P;
    a.G = c->G;
    a.M = c->M;
    a.N = c->N;
    a.K = c->K;
    a.max_iters = c->max_iters;
    return a;
}

// Invert the M x M symmetric matrix sum_i b_i b_i^T (Eq. Zest) by Gauss-Jordan with partial pivoting.
bool invert_gram(const std::vector<double>& basis, int P, int M, std::vector<double>& inv) {
    std::vector<double> a((size_t)M * 2 * M, 0.0);
    double scale = 0.0;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double s = 0.0;
            for (int f = 0; f < P; ++f) s += basis[(size_t)f * M + i] * basis[(size_t)f * M + j];
            a[(size_t)i * 2 * M + j] = s;
            scale = std::max(scale, std::fabs(s));
        }
    for (int i = 0; i < M; ++i) a[(size_t)i * 2 * M + M + i] = 1.0;
    for (int col = 0; col < M; ++col) {
        int piv = col;
        for (int r = col + 1; r < M; ++r)
            if (std::fabs(a[(size_t)r * 2 * M + col]) > std::fabs(a[(size_t)piv * 2 * M + col])) piv = r;
        if (!(std::fabs(a[(size_t)piv * 2 * M + col]) > 1e-13 * scale)) return false;
        if (piv != col)
            for (int j = 0; j < 2 * M; ++j) std::swap(a[(size_t)piv * 2 * M + j], a[(size_t)col * 2 * M + j]);
        const double d = a[(size_t)col * 2 * M + col];
        for (int j = 0; j < 2 * M; ++j) a[(size_t)col * 2 * M + j] /= d;
        for (int r = 0; r < M; ++r) {
            if (r == col) continue;
            const double f = a[(size_t)r * 2 * M + col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * M; ++j) a[(size_t)r * 2 * M + j] -= f * a[(size_t)col * 2 * M + j];
        }
    }
    inv.assign((size_t)M * M, 0.0);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) inv[(size_t)i * M + j] = a[(size_t)i * 2 * M + M + j];
    return true;
}

void free_layout(calib_ctx* c) {
    cudaFree(c->V); c->V = nullptr;
    cudaFree(c->C); c->C = nullptr;
    cudaFree(c->desc); c->desc = nullptr;
    cudaFree(c->slot); c->slot = nullptr;
    cudaFree(c->slot_b); c->slot_b = nullptr;
    cudaFree(c->gw); c->gw = nullptr;
    cudaFree(c->ssU); c->ssU = nullptr;
    cudaFree(c->ssS); c->ssS = nullptr;
}

void clear_graphs(calib_ctx* c) {
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto& pp : kv.second.prof) {
            cudaEventDestroy(pp.a);
            cudaEventDestroy(pp.b);
        }
    }
    c->graphs.clear();
}

// Circulant-diagonal slot layout for the given flags (see calib_internal.cuh).
int build_layout(calib_ctx* c, const uint8_t* flags) {
    const int N = c->N, D = c->D, A = c->A, K = c->K;
    std::vector<int> pair_b((size_t)N * N, -1);
    for (int b = 0; b < c->B; ++b) pair_b[(size_t)c->pq[2 * b] * N + c->pq[2 * b + 1]] = b;
    c->desc_h.assign((size_t)A * D, DiagDesc{});
    c->slot_h.clear();
    c->slot_b_h.clear();
    long long voff = 0, coff = 0;
    const int KK = K * (K + 1) / 2;
    int smax = 4;
    double alg_res = 0, alg_hv = 0, alg_ssh = 0, alg_sst = 0;
    double flo[4] = {0, 0, 0, 0};
    double alg_stp = 0, flo_stp = 0;
    for (int a = 0; a < A; ++a) {
        for (int d = 1; d <= D; ++d) {
            DiagDesc& dd = c->desc_h[(size_t)a * D + d - 1];
            dd.slot_off = (int)c->slot_h.size();
            const int n_i = (2 * d == N) ? N / 2 : N;
            int n = 0;
            for (int i = 0; i < n_i; ++i) {
                const int j = (i + d) % N;
                const int p = std::min(i, j), q = std::max(i, j);
                const int b = pair_b[(size_t)p * N + q];
                if (b < 0) continue;
                if (flags && flags[(size_t)a * c->B + b]) continue;
                const int rev = (i > j) ? 1 : 0;
                c->slot_h.push_back(i | (j << 8) | (rev << 16));
                c->slot_b_h.push_back(b);
                ++n;
            }
            dd.n = n;
            dd.n_pad = (n + 3) / 4 * 4;
            dd.voff = voff;
            dd.coff = coff;
            voff += (long long)c->T[a] * dd.n_pad * 4;
            coff += (long long)c->T[a] * dd.n_pad * K;
            smax = std::max(smax, dd.n_pad);
            alg_res += (double)n * c->T[a] * (32.0 + 8.0 * K);
            alg_hv += (double)n * c->T[a] * (8.0 * K);
            alg_ssh += (double)n * 8.0 * KK;
            alg_sst += (double)n * (32.0 * K + 8.0 * KK);
            // Real flops per baseline (complex multiply 6, complex multiply-add 8, 2x2 complex
            // product 56): P_l / Q_l per direction, the per-sample or S-weighted direction sums,
            // and the two station terms per direction with their accumulation (128).
            const double T = c->T[a];
            flo[0] += (double)n * (T * (64.0 * K + 8.0) + 56.0 * K + 128.0 * K);
            flo[1] += (double)n * (T * 64.0 * K + 120.0 * K + 128.0 * K);
            flo[2] += (double)n * (248.0 * K + 32.0 * K * K);
            flo[3] += (double)n * (432.0 * K + 64.0 * K * K);
            // statistics pass: V and C of every sample read, U and S written; U: 4K and S: KK
            // complex multiply-adds per sample
            alg_stp += (double)n * (T * (32.0 + 8.0 * K) + 32.0 * K + 8.0 * KK);
            flo_stp += (double)n * T * (32.0 * K + 8.0 * KK);
        }
    }
    c->int_v = voff;
    c->int_c = coff;
    // sufficient statistics: full circulant layout, NP positions per (agent, diagonal)
    const long long NP = (N + 3) / 4 * 4;
    c->int_u = (long long)A * D * NP * K * 4;
    c->int_s = (long long)A * D * NP * KK;
    c->slots_max = smax;
    c->alg_bytes[0] = alg_res;
    c->alg_bytes[1] = alg_hv;
    c->alg_bytes[2] = alg_ssh;
    c->alg_bytes[3] = alg_sst;
    for (int i = 0; i < 4; ++i) c->alg_flops[i] = flo[i];
    c->alg_bytes[6] = alg_stp;
    c->alg_flops[6] = flo_stp;
    c->TT_res = sweep_tile_samples(smax, K, false);
    c->TT_hv = sweep_tile_samples(smax, K, true);
    if (sweep_threads(smax) > 512) return fail(CALIB_EINVAL, "too many stations for one CTA per diagonal");
    if ((size_t)3 * 24 * 1024 + sweep_smem_bytes(N, K, true) + 4096 > 200 * 1024)
        return fail(CALIB_EINVAL, "N*K too large for the sweep kernels' shared memory");
    if (c->formulation == 0 && ss_sweep_smem_bytes(N, K, false, nullptr) > 200 * 1024)
        return fail(CALIB_EINVAL, "N*K too large for the statistics sweeps' shared memory; use CALIB_FORM_DIRECT");

    free_layout(c);
    CK(dalloc(&c->V, (size_t)c->int_v));
    CK(dalloc(&c->C, (size_t)c->int_c));
    CK(dalloc(&c->desc, c->desc_h.size()));
    CK(dalloc(&c->slot, c->slot_h.size()));
    CK(dalloc(&c->slot_b, c->slot_b_h.size()));
    CK(dalloc(&c->gw, (size_t)A * K * N * ((N + 3) / 4 * 4)));
    CK(dalloc(&c->ssU, (size_t)c->int_u));
    CK(dalloc(&c->ssS, (size_t)c->int_s));
    // statistics of flagged baselines stay zero: the statistics pass never writes their positions
    CK(cudaMemset(c->ssU, 0, (size_t)std::max(1LL, c->int_u) * sizeof(float2)));
    CK(cudaMemset(c->ssS, 0, (size_t)std::max(1LL, c->int_s) * sizeof(float2)));
    CK(cudaMemcpy(c->desc, c->desc_h.data(), c->desc_h.size() * sizeof(DiagDesc), cudaMemcpyHostToDevice));
    if (!c->slot_h.empty()) {
        CK(cudaMemcpy(c->slot, c->slot_h.data(), c->slot_h.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->slot_b, c->slot_b_h.data(), c->slot_b_h.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    CK(cudaMemset(c->V, 0, (size_t)std::max(1LL, c->int_v) * sizeof(float2)));
    CK(cudaMemset(c->C, 0, (size_t)std::max(1LL, c->int_c) * sizeof(float2)));
    clear_graphs(c);
    c->data_set = false;
    c->coh_set = false;
    c->ss_dirty = true;
    return CALIB_OK;
}

int ensure_staging(calib_ctx* c, size_t bytes) {
    if (c->staging_bytes >= bytes) return CALIB_OK;
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->staging);
    c->staging = nullptr;
    c->staging_bytes = 0;
    CK(cudaMalloc(&c->staging, bytes));
    c->staging_bytes = bytes;
    return CALIB_OK;
}

// Device pointer to caller data: device pointers pass through, host data is copied to staging.
int stage_in(calib_ctx* c, const void* src, size_t bytes, int ptr_kind, const void** dev, size_t staging_off = 0) {
    if (ptr_kind == 1) {
        *dev = src;
        return CALIB_OK;
    }
    int rc = ensure_staging(c, staging_off + bytes);
    if (rc) return rc;
    char* d = static_cast<char*>(c->staging) + staging_off;
    CK(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, c->stream));
    *dev = d;
    return CALIB_OK;
}

int copy_out(calib_ctx* c, void* dst, const void* dev_src, size_t bytes, int ptr_kind) {
    if (!dst) return CALIB_OK;
    CK(cudaMemcpyAsync(dst, dev_src, bytes, ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    return CALIB_OK;
}

int check_status(calib_ctx* c) {
    int st = 0;
    CK(cudaMemcpy(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & STATUS_TIMEOUT) return fail(CALIB_ETIMEOUT, "a bounded in-kernel wait timed out");
    if (st & STATUS_NONFINITE) return fail(CALIB_ENUMERIC, "input data contain non-finite values");
    return CALIB_OK;
}

// ---------------------------------------------------------------------------- schedule

struct Enq {
    calib_ctx* c;
    GraphEntry* ge;
    cudaError_t err = cudaSuccess;
    void ok(cudaError_t e) {
        if (err == cudaSuccess && e != cudaSuccess) err = e;
        ge->kernels += 1;
    }
    // Profiling: CUDA events recorded around a launch of the given kind on the library stream.
    ProfPair begin(int kind) {
        ProfPair pp{};
        if (c->profiling) {
            cudaEventCreate(&pp.a);
            cudaEventCreate(&pp.b);
            pp.kind = kind;
            cudaEventRecordWithFlags(pp.a, c->stream, cudaEventRecordExternal);
        }
        return pp;
    }
    void end(ProfPair& pp) {
        if (c->profiling) {
            cudaEventRecordWithFlags(pp.b, c->stream, cudaEventRecordExternal);
            ge->prof.push_back(pp);
        }
    }
    // the inner solver's per-agent kernels: PCG / LM damping, or truncated CG / trust region
    void cg_step(const LMArgs& la, bool last) {
        ProfPair pp = begin(4);
        ok(c->jupdate == CALIB_JUPDATE_RTR ? launch_tcg_step(la, last, c->stream) : launch_cg_step(la, last, c->stream));
        end(pp);
    }
    void lm_eval(const LMArgs& la, int mode) {
        ProfPair pp = begin(5);
        ok(c->jupdate == CALIB_JUPDATE_RTR ? launch_rtr_eval(la, mode, c->stream) : launch_lm_eval(la, mode, c->stream));
        end(pp);
    }
    void sweep(int mode, const float* J, const float* eta, bool pdl = false) {
        const bool ss = c->formulation == 0 && mode != SWEEP_RESIDUAL;
        ProfPair pp = begin(ss ? (mode == SWEEP_HESSVEC ? 2 : 3) : (mode == SWEEP_HESSVEC ? 1 : 0));
        if (ss) {  // the statistics trial pass takes the trial point J' itself (written by the last PCG step)
            const float* e2 = mode == SWEEP_HESSVEC ? eta : c->Jt;
            const bool hv = mode == SWEEP_HESSVEC;
            SSArgs sa = ss_args(c, J, e2, hv);
            sa.pdl = pdl ? 1 : 0;
            ok(launch_ss_sweep(sa, hv, hv ? c->part_hv.grid : c->part_tr.grid, c->stream));
        } else {
            ok(launch_sweep(sweep_args(c, mode, J, eta), mode, c->stream));
        }
        end(pp);
    }
};

// SAGE J-update (step D1): n_sage sweeps over the directions; direction k's one-direction problem
// (expectation step on the statistics, sage.cu) is solved by n_lm trust-region steps starting from
// the gradient of a trial pass at J' = J; its solution is written back before the next direction.
// Then the whole problem's data cost, gradient and Jacobi blocks at the new J (the records).
void enqueue_sage_jupdate(Enq& q) {
    calib_ctx* c = q.c;
    const SageArgs sg = sage_args(c);
    const SSArgs hv1 = sage_ss_args(c, true), tr1 = sage_ss_args(c, false);
    for (int sweep = 0; sweep < c->n_sage; ++sweep)
        for (int k = 0; k < c->K; ++k) {
            const LMArgs lh = sage_lm_args(c, PARTS_SS_HESSIAN, k), lt = sage_lm_args(c, PARTS_SS_TRIAL, k);
            q.ok(launch_sage_prepare(sg, k, c->stream));
            q.ok(launch_ss_sweep(tr1, false, c->part_tr.grid, c->stream));
            q.ok(launch_rtr_eval(lt, LM_BEGIN_FROM_TRIAL, c->stream));
            for (int l = 0; l < c->n_lm; ++l) {
                for (int j = 0; j < c->n_cg; ++j) {
                    q.ok(launch_ss_sweep(hv1, true, c->part_hv.grid, c->stream));
                    q.ok(launch_tcg_step(lh, j == c->n_cg - 1, c->stream));
                }
                q.ok(launch_ss_sweep(tr1, false, c->part_tr.grid, c->stream));
                q.ok(launch_rtr_eval(lt, LM_ACCEPT, c->stream));
            }
            q.ok(launch_sage_scatter(sg, k, c->stream));
        }
    q.ok(launch_sweep(sweep_args(c, SWEEP_RESIDUAL, c->J, nullptr), SWEEP_RESIDUAL, c->stream));
    q.ok(launch_lm_eval(lm_args(c, PARTS_DIRECT), LM_BEGIN_FROM_PARTIALS, c->stream));
}

void enqueue_iteration(Enq& q, bool eval_first, bool gauge) {
    calib_ctx* c = q.c;
    if (c->jupdate == CALIB_JUPDATE_SAGE) {
        const ConsArgs ca = cons_args(c);
        enqueue_sage_jupdate(q);
        if (gauge) q.ok(launch_gauge(ca, c->stream));
        q.ok(launch_zy_update(ca, c->stream));
        q.ok(launch_records(ca, c->stream));
        return;
    }
    const bool ssf = c->formulation == 0;
    // Programmatic dependent launch through the LM chain (each kernel's prologue overlaps the tail of
    // the one before); not with per-kernel profiling events, whose records sit between the kernels.
    const bool pdl = c->jupdate == CALIB_JUPDATE_LM && !c->profiling;
    LMArgs la_hv = lm_args(c, ssf ? PARTS_SS_HESSIAN : PARTS_DIRECT);  // after a Hessian sweep
    LMArgs la = lm_args(c, ssf ? PARTS_SS_TRIAL : PARTS_DIRECT);       // after the trial sweep
    la_hv.pdl = la.pdl = pdl ? 1 : 0;
    const ConsArgs ca = cons_args(c);
    if (eval_first) {  // the residual sweep is the direct one in both formulations (it yields g exactly)
        q.sweep(SWEEP_RESIDUAL, c->J, nullptr);
        LMArgs l0 = lm_args(c, PARTS_DIRECT);
        l0.pdl = la.pdl;
        q.lm_eval(l0, LM_BEGIN_FROM_PARTIALS);
    } else {
        q.lm_eval(la, LM_BEGIN_REUSE);
    }
    for (int l = 0; l < c->n_lm; ++l) {
        for (int k = 0; k < c->n_cg; ++k) {
            q.sweep(SWEEP_HESSVEC, c->J, c->p, pdl);
            q.cg_step(la_hv, k == c->n_cg - 1);  // the last one forms the trial point
        }
        q.sweep(SWEEP_TRIAL, c->J, c->x, pdl);
        q.lm_eval(la, LM_ACCEPT);
    }
    ProfPair pp = q.begin(7);
    if (gauge) q.ok(launch_gauge(ca, c->stream));
    q.ok(launch_zy_update(ca, c->stream));
    q.ok(launch_records(ca, c->stream));
    q.end(pp);
}

int ensure_stats(calib_ctx* c, int n) {
    if (c->max_iters >= n) return CALIB_OK;
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->stats);
    c->stats = nullptr;
    CK(dalloc(&c->stats, (size_t)n * 4));
    c->max_iters = n;
    clear_graphs(c);  // graphs hold the old pointer and capacity
    return CALIB_OK;
}

bool valid_kind(int k) { return k == 0 || k == 1; }

// Shape class of a tuning result: the timing depends on these alone.
struct TuneKey {
    int N, K, A, D, form, n_cg;
    long long work;  // total slot-samples (direct form) or slots (statistics)
    bool operator<(const TuneKey& o) const {
        return std::tie(N, K, A, D, form, n_cg, work) < std::tie(o.N, o.K, o.A, o.D, o.form, o.n_cg, o.work);
    }
};
struct TuneResult { int hv, tr; };  // split of the Hessian and of the trial pass
std::map<TuneKey, TuneResult>& tune_cache() {
    static std::map<TuneKey, TuneResult> m;
    return m;
}

// Time the two halves of one LM step - n_cg Hessian passes with their PCG steps, and the trial
// pass with its reduction - for each candidate work split and keep the fastest: CTAs per SM of
// each statistics sweep (chosen per pass), or diagonals per CTA of the direct sweeps (one value,
// the fastest whole step). Runs on the context's data; touches only scratch outputs and the PCG
// vectors x, r, p, which the next LM begin re-initialises (the PCG steps run in timing mode and
// write no agent state).
int apply_split(calib_ctx* c, TuneResult v) {
    if (c->formulation == 0) {
        const int rc = set_partition(c, c->part_hv, v.hv);
        return rc ? rc : set_partition(c, c->part_tr, v.tr);
    }
    c->chunk_diags = v.hv;
    c->n_chunks = (c->D + v.hv - 1) / v.hv;
    return CALIB_OK;
}

int autotune(calib_ctx* c) {
    long long work = 0;
    for (const DiagDesc& d : c->desc_h) work += (long long)d.n;
    for (int a = 0; a < c->A && c->formulation == 1; ++a) work += (long long)c->T[a];
    const TuneKey key{c->N, c->K, c->A, c->D, c->formulation, c->n_cg, work};
    auto hit = tune_cache().find(key);
    c->tune_log.clear();
    if (hit != tune_cache().end()) {
        const int rc = apply_split(c, hit->second);
        if (rc) return rc;
        c->tune_pending = false;
        clear_graphs(c);
        return CALIB_OK;
    }
    std::vector<int> cands;
    if (c->formulation == 0) {
        const long long W = (long long)c->A * c->D;
        long long last_grid = -1;
        for (int m : {1, 2, 3, 4, 5, 6, 8, 12, 16, 24}) {
            const long long grid = std::min(W, (long long)c->sms * m);
            if (grid == last_grid) break;  // capped at one item per CTA
            cands.push_back(m);
            last_grid = grid;
        }
    } else {
        for (int cd = 1; cd <= c->D; cd *= 2) cands.push_back(cd);
        if (cands.back() != c->D) cands.push_back(c->D);
    }
    cudaEvent_t e0, e1, e2;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreate(&e2));
    const bool ssf = c->formulation == 0;
    double best_hv = 1e300, best_tr = 1e300, best_sum = 1e300;
    TuneResult best{cands.front(), cands.front()};
    int best_direct = cands.front();
    const int reps = 3;
    for (int v : cands) {
        const int rc = apply_split(c, TuneResult{v, v});
        if (rc) return rc;
        LMArgs la_hv = lm_args(c, ssf ? PARTS_SS_HESSIAN : PARTS_DIRECT);
        LMArgs la_tr = lm_args(c, ssf ? PARTS_SS_TRIAL : PARTS_DIRECT);
        la_hv.timing = 1;
        la_tr.Jt = c->J;
        auto hessian_half = [&]() -> cudaError_t {
            cudaError_t err = cudaSuccess;
            for (int k = 0; k < c->n_cg && err == cudaSuccess; ++k) {
                if (ssf)
                    err = launch_ss_sweep(ss_args(c, c->J, c->p, true), true, c->part_hv.grid, c->stream);
                else
                    err = launch_sweep(sweep_args(c, SWEEP_HESSVEC, c->J, c->p), SWEEP_HESSVEC, c->stream);
                if (err == cudaSuccess) err = launch_cg_step(la_hv, false, c->stream);
            }
            return err;
        };
        auto trial_half = [&]() -> cudaError_t {
            cudaError_t err;
            if (ssf)
                err = launch_ss_sweep(ss_args(c, c->J, c->J, false), false, c->part_tr.grid, c->stream);  // J' = J
            else
                err = launch_sweep(sweep_args(c, SWEEP_TRIAL, c->J, c->x), SWEEP_TRIAL, c->stream);
            return err != cudaSuccess ? err : launch_eval_output(la_tr, c->evOut, c->evL, c->evG, c->stream);
        };
        CK(hessian_half());  // warm
        CK(trial_half());
        CK(cudaEventRecord(e0, c->stream));
        for (int r = 0; r < reps; ++r) CK(hessian_half());
        CK(cudaEventRecord(e1, c->stream));
        for (int r = 0; r < reps; ++r) CK(trial_half());
        CK(cudaEventRecord(e2, c->stream));
        CK(cudaEventSynchronize(e2));
        float ms_hv = 0.f, ms_tr = 0.f;
        CK(cudaEventElapsedTime(&ms_hv, e0, e1));
        CK(cudaEventElapsedTime(&ms_tr, e1, e2));
        ms_hv /= reps;
        ms_tr /= reps;
        c->launches += (long long)(reps + 1) * (2 * c->n_cg + 2);
        c->tune_log.push_back(TuneEntry{v, ms_hv, ms_tr});
        if (ms_hv < best_hv) { best_hv = ms_hv; best.hv = v; }
        if (ms_tr < best_tr) { best_tr = ms_tr; best.tr = v; }
        if (ms_hv + ms_tr < best_sum) { best_sum = ms_hv + ms_tr; best_direct = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (!ssf) best = TuneResult{best_direct, best_direct};
    const int rc = apply_split(c, best);
    if (rc) return rc;
    c->tune_pending = false;
    tune_cache()[key] = best;
    clear_graphs(c);
    return check_status(c);
}

}  // namespace

void calib::set_last_error(const std::string& msg) { g_err = msg; }

extern "C" {

void calib_default_options(calib_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->n_intervals = 1;
    opt->n_samples = 1;
    opt->samples_per_agent = nullptr;
    opt->n_lm = 10;
    opt->n_cg = 4;
    opt->chunk_diagonals = 0;
    opt->cuda_stream = nullptr;
    opt->formulation = CALIB_FORM_STATISTICS;
    opt->ctas_per_sm = 0;
    opt->jupdate = CALIB_JUPDATE_LM;
    opt->n_sage = 1;
    opt->freq_groups = 1;
}

int calib_init(calib_ctx** out, int n_stations, int n_baselines, const int32_t* pq, int n_dirs, int n_freqs,
               const double* freqs_hz, int n_basis, const double* basis, const double* rho,
               const calib_options* opt_in) {
    if (!out) return fail(CALIB_EINVAL, "out is NULL");
    *out = nullptr;
    calib_options opt;
    calib_default_options(&opt);
    if (opt_in) opt = *opt_in;
    const int N = n_stations, B = n_baselines, K = n_dirs, P = n_freqs, M = n_basis;
    if (N < 2 || N > 128) return fail(CALIB_EINVAL, "n_stations must be in [2, 128]");
    if (B < 1 || B > N * (N - 1) / 2) return fail(CALIB_EINVAL, "n_baselines must be in [1, N(N-1)/2]");
    if (K < 1 || K > MAX_K) return fail(CALIB_EINVAL, "n_dirs must be in [1, 16]");
    if (P < 1) return fail(CALIB_EINVAL, "n_freqs must be >= 1");
    if (M < 1 || M > MAX_M) return fail(CALIB_EINVAL, "n_basis must be in [1, 16]");
    if (!pq || !freqs_hz || !basis || !rho) return fail(CALIB_EINVAL, "pq, freqs_hz, basis and rho are required");
    const int G = opt.freq_groups < 1 ? 1 : opt.freq_groups;
    if (P % G != 0) return fail(CALIB_EINVAL, "freq_groups must divide n_freqs");
    if (P / G < M)
        return fail(CALIB_ERANK, "need at least as many frequencies as basis terms in every consensus problem (P >= M; "
                                 "P/G >= M with frequency groups)");
    if (opt.n_intervals < 1) return fail(CALIB_EINVAL, "n_intervals must be >= 1");
    if (opt.n_lm < 1 || opt.n_cg < 1) return fail(CALIB_EINVAL, "n_lm and n_cg must be >= 1");
    if (opt.formulation != CALIB_FORM_STATISTICS && opt.formulation != CALIB_FORM_DIRECT)
        return fail(CALIB_EINVAL, "formulation must be CALIB_FORM_STATISTICS or CALIB_FORM_DIRECT");
    if (opt.jupdate != CALIB_JUPDATE_LM && opt.jupdate != CALIB_JUPDATE_RTR && opt.jupdate != CALIB_JUPDATE_SAGE)
        return fail(CALIB_EINVAL, "jupdate must be CALIB_JUPDATE_LM, CALIB_JUPDATE_RTR or CALIB_JUPDATE_SAGE");
    if (opt.jupdate == CALIB_JUPDATE_SAGE && opt.formulation != CALIB_FORM_STATISTICS)
        return fail(CALIB_EINVAL, "CALIB_JUPDATE_SAGE needs CALIB_FORM_STATISTICS");
    if (opt.jupdate == CALIB_JUPDATE_SAGE && opt.n_sage < 1) return fail(CALIB_EINVAL, "n_sage must be >= 1");
    std::vector<char> seen((size_t)N * N, 0);
    for (int b = 0; b < B; ++b) {
        const int p = pq[2 * b], q = pq[2 * b + 1];
        if (p < 0 || q >= N || p >= q) return fail(CALIB_EINVAL, "each pair must satisfy 0 <= p < q < N");
        if (seen[(size_t)p * N + q]) return fail(CALIB_EINVAL, "duplicate baseline");
        seen[(size_t)p * N + q] = 1;
    }
    for (int k = 0; k < K; ++k)
        if (!(rho[k] > 0.0) || !std::isfinite(rho[k])) return fail(CALIB_EINVAL, "rho must be finite and > 0");
    for (int i = 0; i < P * M; ++i)
        if (!std::isfinite(basis[i])) return fail(CALIB_EINVAL, "basis must be finite");
    const int A = opt.n_intervals * P;
    std::vector<int> T(A);
    for (int a = 0; a < A; ++a) {
        T[a] = opt.samples_per_agent ? opt.samples_per_agent[a] : opt.n_samples;
        if (T[a] < 1) return fail(CALIB_EINVAL, "every agent needs at least one sample");
    }
    // (sum_i b_i b_i^T)^-1 of every frequency group (its interleaved rows g, g + G, ...)
    std::vector<double> Pinv;
    for (int g = 0; g < G; ++g) {
        std::vector<double> rows, inv;
        for (int f = g; f < P; f += G) rows.insert(rows.end(), basis + (size_t)f * M, basis + (size_t)(f + 1) * M);
        if (!invert_gram(rows, P / G, M, inv)) return fail(CALIB_ERANK, "sum_i b_i b_i^T is singular");
        Pinv.insert(Pinv.end(), inv.begin(), inv.end());
    }

    calib_ctx* c = new calib_ctx();
    c->N = N; c->B = B; c->K = K; c->P = P; c->M = M; c->I = opt.n_intervals; c->A = A; c->G = G;
    c->D = N / 2;
    c->n_lm = opt.n_lm;
    c->n_cg = opt.n_cg;
    c->formulation = opt.formulation;
    c->jupdate = opt.jupdate;
    c->n_sage = opt.jupdate == CALIB_JUPDATE_SAGE ? opt.n_sage : 1;
    c->pq.assign(pq, pq + 2 * (size_t)B);
    c->freqs.assign(freqs_hz, freqs_hz + P);
    c->basis.assign(basis, basis + (size_t)P * M);
    c->rho.assign(rho, rho + K);
    c->rho_f.resize(K);
    for (int k = 0; k < K; ++k) c->rho_f[k] = (float)rho[k];
    c->Pinv = Pinv;
    c->T = T;
    c->Tmax = *std::max_element(T.begin(), T.end());
    c->vis_off.resize(A);
    c->coh_off.resize(A);
    long long vo = 0, co = 0;
    for (int a = 0; a < A; ++a) {
        c->vis_off[a] = vo;
        c->coh_off[a] = co;
        vo += (long long)B * T[a] * 4;
        co += (long long)B * T[a] * K;
    }
    c->user_v = vo;
    c->user_c = co;
    // Work split of the sweeps: fixed by the options, else provisional until the autotuner runs.
    if (opt.chunk_diagonals > 0) {
        c->chunk_diags = std::min(opt.chunk_diagonals, c->D);
    } else {
        if (c->formulation == 1) c->tune_pending = true;
        const int want = std::max(1, std::min(c->D, (1216 + A - 1) / A));
        c->chunk_diags = (c->D + want - 1) / want;
    }
    c->n_chunks = (c->D + c->chunk_diags - 1) / c->chunk_diags;
    if (opt.ctas_per_sm > 0) {
        c->part_hv.m = c->part_tr.m = opt.ctas_per_sm;
    } else if (c->formulation == 0) {
        c->tune_pending = true;
    }

    auto bail = [&](int rc) { calib_destroy(c); return rc; };
    if (cudaGetDevice(&c->dev) != cudaSuccess) return bail(fail(CALIB_ECUDA, "no CUDA device"));
    if (opt.cuda_stream) {
        c->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(CALIB_ECUDA, "cudaStreamCreate failed"));
        c->own_stream = true;
    }
    cudaError_t pe = prepare_sweep_kernels();
    if (pe == cudaSuccess) pe = prepare_lm_kernels();
    if (pe == cudaSuccess) pe = prepare_data_kernels();
    if (pe == cudaSuccess) pe = prepare_ss_kernels();
    if (pe != cudaSuccess) return bail(fail(CALIB_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(pe)));

    const size_t vec = (size_t)A * K * N * 8;
    bool okm = true;
    for (float** pp : {&c->J, &c->Jt, &c->Y, &c->BZ, &c->gradg, &c->grad, &c->x, &c->r, &c->p,
                       &c->evJ, &c->evE, &c->evOut})
        okm = okm && dalloc(pp, vec) == cudaSuccess;
    okm = okm && dalloc(&c->Gm, (size_t)A * K * N * 4) == cudaSuccess;
    // partials sized for one diagonal per CTA, the largest chunk count the autotuner may pick
    okm = okm && dalloc(&c->part, (size_t)A * c->D * K * N * 8) == cudaSuccess;
    okm = okm && dalloc(&c->part_cost, (size_t)A * c->D) == cudaSuccess;
    okm = okm && dalloc(&c->part_dcost, (size_t)A * c->D) == cudaSuccess;
    const size_t zs = (size_t)c->I * c->G * K * M * N * 8;
    okm = okm && dalloc(&c->Z, zs) == cudaSuccess && dalloc(&c->Zprev, zs) == cudaSuccess;
    okm = okm && dalloc(&c->basis_d, (size_t)P * M) == cudaSuccess && dalloc(&c->Pinv_d, (size_t)c->G * M * M) == cudaSuccess;
    okm = okm && dalloc(&c->freqs_d, (size_t)P) == cudaSuccess && dalloc(&c->rho_d, (size_t)K) == cudaSuccess;
    okm = okm && dalloc(&c->st, (size_t)A) == cudaSuccess && dalloc(&c->prim, (size_t)A * K) == cudaSuccess;
    okm = okm && dalloc(&c->dual2, (size_t)c->I * c->G * K * Z_SLOTS) == cudaSuccess;
    okm = okm && dalloc(&c->basis_df, (size_t)P * M) == cudaSuccess && dalloc(&c->Pinv_df, (size_t)c->G * M * M) == cudaSuccess &&
          dalloc(&c->rinv_df, (size_t)K) == cudaSuccess;
    okm = okm && dalloc(&c->prim_part, (size_t)A * K * Z_SLOTS) == cudaSuccess &&
          dalloc(&c->pen_part, (size_t)A * K * Z_SLOTS) == cudaSuccess;
    okm = okm && dalloc(&c->rec_part, (size_t)(A + REC_AGENTS - 1) / REC_AGENTS * 3) == cudaSuccess &&
          dalloc(&c->rec_count, 1) == cudaSuccess;
    okm = okm && dalloc(&c->iter_counter, 1) == cudaSuccess && dalloc(&c->status, 1) == cudaSuccess;
    okm = okm && dalloc(&c->evL, (size_t)A) == cudaSuccess && dalloc(&c->evG, (size_t)A) == cudaSuccess;
    okm = okm && dalloc(&c->T_d, (size_t)A) == cudaSuccess && dalloc(&c->part_hv.pn, (size_t)A) == cudaSuccess &&
          dalloc(&c->part_tr.pn, (size_t)A) == cudaSuccess;
    okm = okm && dalloc(&c->vis_off_d, (size_t)A) == cudaSuccess && dalloc(&c->coh_off_d, (size_t)A) == cudaSuccess;
    if (c->jupdate == CALIB_JUPDATE_SAGE) {
        const size_t npos = (size_t)A * c->D * ((N + 3) / 4 * 4), v1 = (size_t)A * N * 8;
        okm = okm && dalloc(&c->sgU, npos * 4) == cudaSuccess && dalloc(&c->sgS, npos) == cudaSuccess;
        for (float** pp : {&c->sgJ, &c->sgJt, &c->sgY, &c->sgBZ, &c->sgGradg, &c->sgGrad, &c->sgX, &c->sgR, &c->sgP})
            okm = okm && dalloc(pp, v1) == cudaSuccess;
        okm = okm && dalloc(&c->sgGm, (size_t)A * N * 4) == cudaSuccess && dalloc(&c->sgSt, (size_t)A) == cudaSuccess;
        if (okm) cudaMemset(c->sgSt, 0, (size_t)A * sizeof(AgentState));
    }
    if (!okm) return bail(fail(CALIB_ENOMEM, "device allocation failed"));
    if (ensure_stats(c, 64) != CALIB_OK) return bail(CALIB_ENOMEM);
    cudaMemcpy(c->basis_d, c->basis.data(), c->basis.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->Pinv_d, c->Pinv.data(), c->Pinv.size() * sizeof(double), cudaMemcpyHostToDevice);
    {
        std::vector<float2> bdf(c->basis.size()), pdf(c->Pinv.size()), rdf(K);
        for (size_t i = 0; i < bdf.size(); ++i) bdf[i] = df_split(c->basis[i]);
        for (size_t i = 0; i < pdf.size(); ++i) pdf[i] = df_split(c->Pinv[i]);
        for (int k = 0; k < K; ++k) rdf[k] = df_split(1.0 / (double)c->rho_f[k]);
        cudaMemcpy(c->basis_df, bdf.data(), bdf.size() * sizeof(float2), cudaMemcpyHostToDevice);
        cudaMemcpy(c->Pinv_df, pdf.data(), pdf.size() * sizeof(float2), cudaMemcpyHostToDevice);
        cudaMemcpy(c->rinv_df, rdf.data(), rdf.size() * sizeof(float2), cudaMemcpyHostToDevice);
        cudaMemset(c->rec_count, 0, sizeof(int));
    }
    cudaMemcpy(c->freqs_d, c->freqs.data(), c->freqs.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(c->rho_d, c->rho_f.data(), c->rho_f.size() * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemcpy(c->T_d, c->T.data(), c->T.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(c->vis_off_d, c->vis_off.data(), c->vis_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    cudaMemcpy(c->coh_off_d, c->coh_off.data(), c->coh_off.size() * sizeof(long long), cudaMemcpyHostToDevice);
    cudaMemset(c->status, 0, sizeof(int));
    cudaMemset(c->st, 0, (size_t)A * sizeof(AgentState));
    cudaMemset(c->prim, 0, (size_t)A * K * sizeof(double));
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess || c->sms < 1)
        return bail(fail(CALIB_ECUDA, "cannot read the SM count"));
    int rc = build_layout(c, nullptr);
    if (rc) return bail(rc);
    rc = set_partition(c, c->part_hv, c->part_hv.m);
    if (rc == CALIB_OK) rc = set_partition(c, c->part_tr, c->part_tr.m);
    if (rc) return bail(rc);
    rc = calib_reset(c);
    if (rc) return bail(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(fail(CALIB_ECUDA, "initialisation failed"));
    *out = c;
    return CALIB_OK;
}

int calib_reset(calib_ctx* c) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    const size_t vec = (size_t)c->A * c->K * c->N * 8;
    CK(launch_identity(c->J, (long long)c->A * c->K * c->N, c->stream));
    CK(cudaMemsetAsync(c->Y, 0, vec * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->BZ, 0, vec * sizeof(float), c->stream));
    const size_t zs = (size_t)c->I * c->G * c->K * c->M * c->N * 8;
    CK(cudaMemsetAsync(c->Z, 0, zs * sizeof(double), c->stream));
    CK(cudaMemsetAsync(c->Zprev, 0, zs * sizeof(double), c->stream));
    c->launches += 1;
    c->cold = true;
    c->need_eval = true;
    c->iters_done = 0;
    return CALIB_OK;
}

int calib_set_data(calib_ctx* c, const void* vis, const void* coh, const uint8_t* flags, int ptr_kind) {
    if (!c || !vis) return fail(CALIB_EINVAL, "ctx and vis are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (flags) {
        std::vector<uint8_t> fh((size_t)c->A * c->B);
        CK(cudaMemcpy(fh.data(), flags, fh.size(), ptr_kind == 1 ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
        if (fh != c->flags_h) {
            CK(cudaStreamSynchronize(c->stream));
            int rc = build_layout(c, fh.data());
            if (rc) return rc;
            c->flags_h = fh;
        }
    }
    IngestArgs ia{};
    ia.desc = c->desc;
    ia.slot = c->slot;
    ia.slot_b = c->slot_b;
    ia.T = c->T_d;
    ia.A = c->A;
    ia.D = c->D;
    ia.K = c->K;
    const void* dv = nullptr;
    int rc = stage_in(c, vis, (size_t)c->user_v * sizeof(float2), ptr_kind, &dv);
    if (rc) return rc;
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    CK(launch_check_finite(static_cast<const float*>(dv), c->user_v * 2, c->status, c->stream));
    ia.src = static_cast<const float2*>(dv);
    ia.src_off = c->vis_off_d;
    ia.dst = c->V;
    ia.is_vis = 1;
    CK(launch_ingest(ia, c->stream));
    c->launches += 2;
    c->ss_dirty = true;
    if (coh) {
        const void* dc = nullptr;
        rc = stage_in(c, coh, (size_t)c->user_c * sizeof(float2), ptr_kind, &dc);
        if (rc) return rc;
        CK(launch_check_finite(static_cast<const float*>(dc), c->user_c * 2, c->status, c->stream));
        ia.src = static_cast<const float2*>(dc);
        ia.src_off = c->coh_off_d;
        ia.dst = c->C;
        ia.is_vis = 0;
        CK(launch_ingest(ia, c->stream));
        CK(launch_gram_weights(c->C, c->desc, c->slot, c->T_d, c->gw, c->A, c->D, c->K, c->N, c->stream));
        c->launches += 3;
        c->coh_set = true;
    }
    c->data_set = true;
    c->need_eval = true;
    if (ptr_kind == 0) {
        CK(cudaStreamSynchronize(c->stream));
        const int rc_st = check_status(c);
        if (rc_st != CALIB_OK) {  // rejected data are not usable: the caller must set them again
            c->data_set = false;
            if (coh) c->coh_set = false;
        }
        return rc_st;
    }
    return CALIB_OK;
}

int calib_predict(calib_ctx* c, const double* uvw_m, const double* sky, int n_src, double f0_hz, int ptr_kind) {
    if (!c || !uvw_m || !sky) return fail(CALIB_EINVAL, "ctx, uvw_m and sky are required");
    if (n_src < 1) return fail(CALIB_EINVAL, "n_src must be >= 1");
    if (!(f0_hz > 0)) return fail(CALIB_EINVAL, "f0_hz must be > 0");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    const int Tmax = *std::max_element(c->T.begin(), c->T.end());
    const size_t ub = (size_t)c->I * Tmax * c->N * 3 * sizeof(double);
    const size_t sb = (size_t)c->K * n_src * 4 * sizeof(double);
    const void *du = nullptr, *ds = nullptr;
    const size_t sky_off = (ub + 255) / 256 * 256;
    if (ptr_kind == 0) {  // size the staging buffer once: a later resize would free the staged uvw
        int rc0 = ensure_staging(c, sky_off + sb);
        if (rc0) return rc0;
    }
    int rc = stage_in(c, uvw_m, ub, ptr_kind, &du, 0);
    if (rc) return rc;
    rc = stage_in(c, sky, sb, ptr_kind, &ds, sky_off);
    if (rc) return rc;
    PredictArgs pa{};
    pa.uvw = static_cast<const double*>(du);
    pa.sky = static_cast<const double*>(ds);
    pa.freqs = c->freqs_d;
    pa.f0 = f0_hz;
    pa.C = c->C;
    pa.desc = c->desc;
    pa.slot = c->slot;
    pa.T = c->T_d;
    pa.A = c->A;
    pa.P = c->P;
    pa.N = c->N;
    pa.K = c->K;
    pa.S = n_src;
    pa.D = c->D;
    pa.Tmax = Tmax;
    CK(launch_predict(pa, c->stream));
    CK(launch_gram_weights(c->C, c->desc, c->slot, c->T_d, c->gw, c->A, c->D, c->K, c->N, c->stream));
    c->launches += 2;
    c->ss_dirty = true;
    c->coh_set = true;
    c->need_eval = true;
    if (ptr_kind == 0) CK(cudaStreamSynchronize(c->stream));
    return CALIB_OK;
}

int calib_get_coherencies(calib_ctx* c, void* coh, int ptr_kind) {
    if (!c || !coh) return fail(CALIB_EINVAL, "ctx and coh are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (!c->coh_set) return fail(CALIB_ESTATE, "no coherencies set or predicted yet");
    const size_t bytes = (size_t)c->user_c * sizeof(float2);
    void* dst = coh;
    if (ptr_kind == 0) {
        int rc = ensure_staging(c, bytes);
        if (rc) return rc;
        dst = c->staging;
    }
    CK(cudaMemsetAsync(dst, 0, bytes, c->stream));
    IngestArgs ia{};
    ia.desc = c->desc;
    ia.slot = c->slot;
    ia.slot_b = c->slot_b;
    ia.T = c->T_d;
    ia.A = c->A;
    ia.D = c->D;
    ia.K = c->K;
    ia.src_off = c->coh_off_d;
    ia.dst = c->C;
    CK(launch_extract_coh(ia, static_cast<float2*>(dst), c->stream));
    c->launches += 1;
    if (ptr_kind == 0) {
        CK(cudaMemcpyAsync(coh, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return CALIB_OK;
}

int calib_residual(calib_ctx* c, const int32_t* subtract, int correct_dir, void* out, int ptr_kind) {
    if (!c || !out) return fail(CALIB_EINVAL, "ctx and out are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (correct_dir < -1 || correct_dir >= c->K) return fail(CALIB_EINVAL, "correct_dir must be -1 or in [0, K)");
    if (!c->data_set || !c->coh_set) return fail(CALIB_ESTATE, "visibilities and coherencies must be set first");
    unsigned mask = 0;
    for (int k = 0; k < c->K; ++k)
        if (!subtract || subtract[k]) mask |= 1u << k;
    const size_t bytes = (size_t)c->user_v * sizeof(float2);
    void* dst = out;
    if (ptr_kind == 0) {
        int rc = ensure_staging(c, bytes);
        if (rc) return rc;
        dst = c->staging;
    }
    // flagged baselines have no slot in the layout: zero them (every output when any is flagged)
    if (std::any_of(c->flags_h.begin(), c->flags_h.end(), [](uint8_t f) { return f != 0; }))
        CK(cudaMemsetAsync(dst, 0, bytes, c->stream));
    ResidualArgs ra{};
    ra.V = c->V;
    ra.C = c->C;
    ra.J = c->J;
    ra.out = static_cast<float2*>(dst);
    ra.vis_off = c->vis_off_d;
    ra.desc = c->desc;
    ra.slot = c->slot;
    ra.slot_b = c->slot_b;
    ra.T = c->T_d;
    ra.A = c->A;
    ra.D = c->D;
    ra.K = c->K;
    ra.N = c->N;
    ra.mask = mask;
    ra.correct = correct_dir;
    CK(launch_residual(ra, c->stream));
    c->launches += 1;
    if (ptr_kind == 0) {
        CK(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return CALIB_OK;
}

int calib_set_initial(calib_ctx* c, const void* J0, int ptr_kind) {
    if (!c || !J0) return fail(CALIB_EINVAL, "ctx and J0 are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    const size_t bytes = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    CK(cudaMemcpyAsync(c->J, J0, bytes, ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    c->need_eval = true;
    if (ptr_kind == 0) CK(cudaStreamSynchronize(c->stream));
    return CALIB_OK;
}

int calib_set_consensus(calib_ctx* c, const void* Zin, const void* Yin, int ptr_kind) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    const cudaMemcpyKind kind = ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t zs = (size_t)c->I * c->G * c->K * c->M * c->N * 8 * sizeof(double);
    const size_t ys = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    if (Zin) CK(cudaMemcpyAsync(c->Z, Zin, zs, kind, c->stream));
    else CK(cudaMemsetAsync(c->Z, 0, zs, c->stream));
    CK(cudaMemcpyAsync(c->Zprev, c->Z, zs, cudaMemcpyDeviceToDevice, c->stream));
    if (Yin) CK(cudaMemcpyAsync(c->Y, Yin, ys, kind, c->stream));
    else CK(cudaMemsetAsync(c->Y, 0, ys, c->stream));
    ConsArgs ca = cons_args(c);
    ca.prim = nullptr;
    CK(launch_bz_only(ca, c->stream));
    c->launches += 1;
    c->cold = false;
    c->iters_done = 0;
    c->need_eval = true;
    if (ptr_kind == 0) CK(cudaStreamSynchronize(c->stream));
    return CALIB_OK;
}

int calib_admm_iter(calib_ctx* c, int n_iters, calib_stats* hist) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    if (n_iters < 1) return fail(CALIB_EINVAL, "n_iters must be >= 1");
    if (!c->data_set || !c->coh_set) return fail(CALIB_ESTATE, "set visibilities and coherencies first");
    int rc = ensure_stats(c, n_iters);
    if (rc) return rc;
    CK(cudaMemsetAsync(c->iter_counter, 0, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    if (c->formulation == 0 && c->ss_dirty) {
        cudaEvent_t p0 = nullptr, p1 = nullptr;
        if (c->profiling) {
            CK(cudaEventCreate(&p0));
            CK(cudaEventCreate(&p1));
            CK(cudaEventRecord(p0, c->stream));
        }
        CK(launch_ss_stats(c->V, c->C, c->ssU, c->ssS, c->desc, c->slot, c->T_d, c->A, c->D, c->K, c->N, c->Tmax, c->status, c->stream));
        if (c->profiling) {
            CK(cudaEventRecord(p1, c->stream));
            CK(cudaEventSynchronize(p1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, p0, p1));
            c->prof_ms[6] += ms;
            c->prof_n[6] += 1;
            cudaEventDestroy(p0);
            cudaEventDestroy(p1);
        }
        c->launches += 1;
        c->ss_dirty = false;
    }
    if (c->tune_pending) {
        rc = autotune(c);
        if (rc) return rc;
        CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    }
    const auto key = std::make_tuple(n_iters, c->need_eval ? 1 : 0, c->cold ? 1 : 0, c->profiling ? 1 : 0);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        GraphEntry ge;
        Enq q{c, &ge};
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        for (int n = 0; n < n_iters; ++n) enqueue_iteration(q, n == 0 && c->need_eval, n == 0 && c->cold);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
        if (q.err != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(CALIB_ECUDA, std::string("kernel launch during capture: ") + cudaGetErrorString(q.err));
        }
        CK(ce);
        cudaError_t ie = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        CK(ie);
        it = c->graphs.emplace(key, ge).first;
    }
    CK(cudaGraphLaunch(it->second.exec, c->stream));
    c->launches += it->second.kernels;
    c->need_eval = false;
    c->cold = false;
    c->iters_done += n_iters;
    CK(cudaStreamSynchronize(c->stream));
    rc = check_status(c);
    if (rc) return rc;
    if (c->profiling) {
        for (auto& pp : it->second.prof) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, pp.a, pp.b));
            c->prof_ms[pp.kind] += ms;
            c->prof_n[pp.kind] += 1;
        }
    }
    if (hist) {
        std::vector<double> h((size_t)n_iters * 4);
        CK(cudaMemcpy(h.data(), c->stats, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < n_iters; ++i) {
            hist[i].primal = h[(size_t)i * 4 + 0];
            hist[i].dual = h[(size_t)i * 4 + 1];
            hist[i].objective = h[(size_t)i * 4 + 2];
            hist[i].resid_norm = h[(size_t)i * 4 + 3];
        }
    }
    return CALIB_OK;
}

namespace {

// Checkpoint blob: a fixed header, then the device arrays in a fixed order (each starting on a
// 64-byte boundary of the blob). Everything a following calib_admm_iter reads from the previous
// one is here, so a resume continues with the same bits.
struct StateHeader {
    char magic[8];          // "CALIBST1"
    int32_t version;        // 1
    int32_t N, B, K, P, M, I, A, formulation, G;
    int32_t cold;           // the next iteration applies the first-iteration gauge projection
    int32_t need_eval;      // the next iteration starts with a residual sweep at J
    int64_t iters_done;     // C-ADMM iterations since the last cold start or warm state
    uint64_t pair_hash;     // FNV-1a of the station pairs and the flags: the data layout
    int64_t total_bytes;
};

uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

uint64_t layout_hash(calib_ctx* c) {
    uint64_t h = fnv1a(c->pq.data(), c->pq.size() * sizeof(int32_t), 1469598103934665603ull);
    h = fnv1a(c->T.data(), c->T.size() * sizeof(int), h);
    return c->flags_h.empty() ? h : fnv1a(c->flags_h.data(), c->flags_h.size(), h);
}

struct StatePart { void* dev; size_t bytes; };

std::vector<StatePart> state_parts(calib_ctx* c) {
    const size_t vb = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    const size_t gb = (size_t)c->A * c->K * c->N * 4 * sizeof(float);
    const size_t zb = (size_t)c->I * c->G * c->K * c->M * c->N * 8 * sizeof(double);
    return {{c->J, vb}, {c->Y, vb}, {c->BZ, vb}, {c->gradg, vb}, {c->Gm, gb},
            {c->Z, zb}, {c->Zprev, zb}, {c->st, (size_t)c->A * sizeof(AgentState)}};
}

size_t round64(size_t x) { return (x + 63) / 64 * 64; }

size_t state_bytes(calib_ctx* c) {
    size_t n = round64(sizeof(StateHeader));
    for (const StatePart& sp : state_parts(c)) n += round64(sp.bytes);
    return n;
}

}  // namespace

int calib_get_state(calib_ctx* c, void* buf, size_t* len) {
    if (!c || !len) return fail(CALIB_EINVAL, "ctx and len are required");
    const size_t need = state_bytes(c);
    if (!buf) {
        *len = need;
        return CALIB_OK;
    }
    if (*len < need) {
        *len = need;
        return fail(CALIB_EINVAL, "state buffer too small (*len now holds the size needed)");
    }
    StateHeader h{};
    std::memcpy(h.magic, "CALIBST1", 8);
    h.version = 1;
    h.N = c->N; h.B = c->B; h.K = c->K; h.P = c->P; h.M = c->M; h.I = c->I; h.A = c->A;
    h.formulation = c->formulation;
    h.G = c->G;
    h.cold = c->cold ? 1 : 0;
    h.need_eval = c->need_eval ? 1 : 0;
    h.iters_done = c->iters_done;
    h.pair_hash = layout_hash(c);
    h.total_bytes = (int64_t)need;
    unsigned char* out = static_cast<unsigned char*>(buf);
    std::memset(out, 0, need);
    std::memcpy(out, &h, sizeof(h));
    size_t off = round64(sizeof(StateHeader));
    for (const StatePart& sp : state_parts(c)) {
        CK(cudaMemcpyAsync(out + off, sp.dev, sp.bytes, cudaMemcpyDeviceToHost, c->stream));
        off += round64(sp.bytes);
    }
    CK(cudaStreamSynchronize(c->stream));
    *len = need;
    return CALIB_OK;
}

int calib_set_state(calib_ctx* c, const void* buf, size_t len) {
    if (!c || !buf) return fail(CALIB_EINVAL, "ctx and buf are required");
    StateHeader h{};
    if (len < sizeof(h)) return fail(CALIB_EINVAL, "state blob too short");
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "CALIBST1", 8) != 0 || h.version != 1)
        return fail(CALIB_EINVAL, "not a calibration state blob (magic or version)");
    if (h.N != c->N || h.B != c->B || h.K != c->K || h.P != c->P || h.M != c->M || h.I != c->I || h.A != c->A ||
        h.formulation != c->formulation || h.G != c->G)
        return fail(CALIB_EINVAL, "state blob was saved for another problem shape or formulation");
    if (h.pair_hash != layout_hash(c))
        return fail(CALIB_EINVAL, "state blob was saved for other station pairs, samples or flags");
    const size_t need = state_bytes(c);
    if ((size_t)h.total_bytes != need || len < need) return fail(CALIB_EINVAL, "state blob has the wrong size");
    const unsigned char* in = static_cast<const unsigned char*>(buf);
    size_t off = round64(sizeof(StateHeader));
    for (const StatePart& sp : state_parts(c)) {
        CK(cudaMemcpyAsync(sp.dev, in + off, sp.bytes, cudaMemcpyHostToDevice, c->stream));
        off += round64(sp.bytes);
    }
    CK(cudaStreamSynchronize(c->stream));
    c->cold = h.cold != 0;
    c->need_eval = h.need_eval != 0;
    c->iters_done = h.iters_done;
    return CALIB_OK;
}

int calib_get_solutions(calib_ctx* c, void* J, void* Zo, void* Yo, int ptr_kind) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    const size_t vb = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    const size_t zb = (size_t)c->I * c->G * c->K * c->M * c->N * 8 * sizeof(double);
    int rc;
    if ((rc = copy_out(c, J, c->J, vb, ptr_kind))) return rc;
    if ((rc = copy_out(c, Zo, c->Z, zb, ptr_kind))) return rc;
    if ((rc = copy_out(c, Yo, c->Y, vb, ptr_kind))) return rc;
    if (ptr_kind == 0) CK(cudaStreamSynchronize(c->stream));
    return CALIB_OK;
}

int calib_get_agent_objective(calib_ctx* c, double* L, double* g) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    std::vector<AgentState> s(c->A);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(s.data(), c->st, s.size() * sizeof(AgentState), cudaMemcpyDeviceToHost));
    for (int a = 0; a < c->A; ++a) {
        if (L) L[a] = s[a].L;
        if (g) g[a] = s[a].g;
    }
    return CALIB_OK;
}

int calib_eval(calib_ctx* c, const void* Jin, double* L, double* g, void* grad, int ptr_kind) {
    if (!c || !Jin) return fail(CALIB_EINVAL, "ctx and J are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (!c->data_set || !c->coh_set) return fail(CALIB_ESTATE, "set visibilities and coherencies first");
    const size_t vb = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    CK(cudaMemcpyAsync(c->evJ, Jin, vb, ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    CK(launch_sweep(sweep_args(c, SWEEP_RESIDUAL, c->evJ, nullptr), SWEEP_RESIDUAL, c->stream));
    LMArgs la = lm_args(c, PARTS_DIRECT);
    la.Jt = c->evJ;
    CK(launch_eval_output(la, c->evOut, c->evL, c->evG, c->stream));
    c->launches += 2;
    int rc;
    if (grad && (rc = copy_out(c, grad, c->evOut, vb, ptr_kind))) return rc;
    if (L && (rc = copy_out(c, L, c->evL, (size_t)c->A * sizeof(double), ptr_kind))) return rc;
    if (g && (rc = copy_out(c, g, c->evG, (size_t)c->A * sizeof(double), ptr_kind))) return rc;
    if (ptr_kind == 0) {
        CK(cudaStreamSynchronize(c->stream));
        return check_status(c);
    }
    return CALIB_OK;
}

int calib_hessvec(calib_ctx* c, const void* Jin, const void* eta, void* out, int ptr_kind) {
    if (!c || !Jin || !eta || !out) return fail(CALIB_EINVAL, "ctx, J, eta and out are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (!c->coh_set) return fail(CALIB_ESTATE, "set coherencies first");
    const size_t vb = (size_t)c->A * c->K * c->N * 8 * sizeof(float);
    const cudaMemcpyKind kind = ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->evJ, Jin, vb, kind, c->stream));
    CK(cudaMemcpyAsync(c->evE, eta, vb, kind, c->stream));
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    CK(launch_sweep(sweep_args(c, SWEEP_HESSVEC, c->evJ, c->evE), SWEEP_HESSVEC, c->stream));
    LMArgs la = lm_args(c, PARTS_DIRECT);
    la.p = c->evE;
    CK(launch_hv_output(la, c->evOut, c->stream));
    c->launches += 2;
    int rc = copy_out(c, out, c->evOut, vb, ptr_kind);
    if (rc) return rc;
    if (ptr_kind == 0) {
        CK(cudaStreamSynchronize(c->stream));
        return check_status(c);
    }
    return CALIB_OK;
}

int calib_sync(calib_ctx* c) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    CK(cudaStreamSynchronize(c->stream));
    return check_status(c);
}

int calib_profile_enable(calib_ctx* c, int on) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    c->profiling = on != 0;
    for (int i = 0; i < calib_ctx::PROF_KINDS; ++i) {
        c->prof_ms[i] = 0.0;
        c->prof_n[i] = 0;
    }
    return CALIB_OK;
}

int calib_profile_read(calib_ctx* c, int cap, const char** names, double* total_ms, long long* launches,
                       double* bytes_per_launch, double* flops_per_launch) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    static const char* kNames[calib_ctx::PROF_KINDS] = {"sweep_residual", "sweep_hessvec", "stats_hessvec",
                                                          "stats_trial", "pcg_step", "lm_eval", "stats_pass",
                                                          "consensus"};
    for (int i = 0; i < calib_ctx::PROF_KINDS && i < cap; ++i) {
        if (names) names[i] = kNames[i];
        if (total_ms) total_ms[i] = c->prof_ms[i];
        if (launches) launches[i] = c->prof_n[i];
        if (bytes_per_launch) bytes_per_launch[i] = c->alg_bytes[i];
        if (flops_per_launch) flops_per_launch[i] = c->alg_flops[i];
    }
    return calib_ctx::PROF_KINDS;
}

long long calib_launch_count(calib_ctx* c) { return c ? c->launches : 0; }

int calib_get_features(calib_ctx* c, float* X, int ptr_kind) {
    if (!c || !X) return fail(CALIB_EINVAL, "ctx and X are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    const size_t rows = (size_t)c->A * c->K * c->N;
    if (!c->xf_d) {
        if (dalloc(&c->xf_d, (size_t)c->A) != cudaSuccess) return fail(CALIB_ENOMEM, "frequency buffer");
        std::vector<double> xf(c->A);
        const double fmin = *std::min_element(c->freqs.begin(), c->freqs.end());
        const double fmax = *std::max_element(c->freqs.begin(), c->freqs.end());
        for (int a = 0; a < c->A; ++a) xf[a] = fmax > fmin ? (c->freqs[a % c->P] - fmin) / (fmax - fmin) : 0.0;
        CK(cudaMemcpy(c->xf_d, xf.data(), xf.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    float* dst = X;
    if (ptr_kind == 0) {
        int rc = ensure_staging(c, rows * 17 * sizeof(float));
        if (rc) return rc;
        dst = static_cast<float*>(c->staging);
    }
    CK(launch_ws_features(c->J, c->BZ, c->xf_d, c->K, c->N, (long long)rows, dst, c->stream));
    c->launches += 1;
    if (ptr_kind == 0) {
        CK(cudaMemcpyAsync(X, dst, rows * 17 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return CALIB_OK;
}

int calib_warm_start(calib_ctx* c, calib_mlp* mlp, const void* J_prev, const void* Z_prev, int* chose, int ptr_kind) {
    if (!c || !J_prev || !Z_prev) return fail(CALIB_EINVAL, "ctx, J_prev and Z_prev are required");
    if (!valid_kind(ptr_kind)) return fail(CALIB_EINVAL, "ptr_kind must be 0 (host) or 1 (device)");
    if (!c->data_set || !c->coh_set) return fail(CALIB_ESTATE, "set visibilities and coherencies first");
    const size_t vec = (size_t)c->A * c->K * c->N * 8;
    if (!c->ws_prev) {
        bool ok = dalloc(&c->ws_prev, vec) == cudaSuccess && dalloc(&c->ws_mlp, vec) == cudaSuccess &&
                  dalloc(&c->ws_L, 2 * (size_t)c->A) == cudaSuccess && dalloc(&c->ws_chose, (size_t)c->A) == cudaSuccess;
        if (!c->xf_d) ok = ok && dalloc(&c->xf_d, (size_t)c->A) == cudaSuccess;
        if (!ok) return fail(CALIB_ENOMEM, "warm-start buffers");
        std::vector<double> xf(c->A);
        const double fmin = *std::min_element(c->freqs.begin(), c->freqs.end());
        const double fmax = *std::max_element(c->freqs.begin(), c->freqs.end());
        for (int a = 0; a < c->A; ++a) xf[a] = fmax > fmin ? (c->freqs[a % c->P] - fmin) / (fmax - fmin) : 0.0;
        CK(cudaMemcpy(c->xf_d, xf.data(), xf.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    // consensus from the previous interval (warm: no first-iteration projection), Y = 0
    int rc = calib_set_consensus(c, Z_prev, nullptr, ptr_kind);
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->ws_prev, J_prev, vec * sizeof(float),
                       ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    if (mlp) {
        CK(mlp_warm_rows(mlp, c->ws_prev, c->BZ, c->xf_d, c->K, c->N, c->A, c->ws_mlp, c->stream));
        LMArgs la = lm_args(c, PARTS_DIRECT);
        const float* starts[2] = {c->ws_mlp, c->ws_prev};
        for (int i = 0; i < 2; ++i) {
            CK(launch_sweep(sweep_args(c, SWEEP_RESIDUAL, starts[i], nullptr), SWEEP_RESIDUAL, c->stream));
            la.Jt = const_cast<float*>(starts[i]);
            CK(launch_eval_output(la, c->evOut, c->ws_L + (size_t)i * c->A, nullptr, c->stream));
        }
        CK(mlp_warm_select(c->ws_mlp, c->ws_prev, c->ws_L, c->ws_L + c->A, c->K * c->N * 8, c->A, c->J, c->ws_chose,
                           c->stream));
        c->launches += 7;
        if (chose) CK(cudaMemcpyAsync(chose, c->ws_chose, (size_t)c->A * sizeof(int),
                                      ptr_kind == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    } else {
        CK(cudaMemcpyAsync(c->J, c->ws_prev, vec * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
        if (chose) {
            if (ptr_kind == 1) CK(cudaMemsetAsync(chose, 0, (size_t)c->A * sizeof(int), c->stream));
            else std::fill(chose, chose + c->A, 0);
        }
    }
    c->need_eval = true;
    c->cold = false;
    c->iters_done = 0;
    if (ptr_kind == 0) CK(cudaStreamSynchronize(c->stream));
    return CALIB_OK;
}

int calib_autotune(calib_ctx* c, int* split, int* split_trial, int cap, int* cand, double* ms_hessian,
                   double* ms_trial, int* n_cand) {
    if (!c) return fail(CALIB_EINVAL, "ctx is NULL");
    if (!c->data_set || !c->coh_set) return fail(CALIB_ESTATE, "set visibilities and coherencies first");
    if (c->formulation == 0 && c->ss_dirty) {
        CK(launch_ss_stats(c->V, c->C, c->ssU, c->ssS, c->desc, c->slot, c->T_d, c->A, c->D, c->K, c->N, c->Tmax, c->status, c->stream));
        c->launches += 1;
        c->ss_dirty = false;
    }
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    tune_cache().clear();
    const int rc = autotune(c);
    if (rc) return rc;
    if (split) *split = c->formulation == 0 ? c->part_hv.m : c->chunk_diags;
    if (split_trial) *split_trial = c->formulation == 0 ? c->part_tr.m : c->chunk_diags;
    const int n = (int)c->tune_log.size();
    for (int i = 0; i < n && i < cap; ++i) {
        if (cand) cand[i] = c->tune_log[i].v;
        if (ms_hessian) ms_hessian[i] = c->tune_log[i].hv;
        if (ms_trial) ms_trial[i] = c->tune_log[i].tr;
    }
    if (n_cand) *n_cand = n;
    return CALIB_OK;
}

int calib_selftest_bounded_wait(int complete_phase, double* elapsed_ms, void* cuda_stream) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int* status = nullptr;
    if (dalloc(&status, 1) != cudaSuccess) return fail(CALIB_ENOMEM, "status word");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int h = 0;
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 128, 0, st>>>(complete_phase != 0, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(status);
    if (e != cudaSuccess) return fail(CALIB_ECUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
    if (elapsed_ms) *elapsed_ms = ms;
    if (h & STATUS_TIMEOUT) return fail(CALIB_ETIMEOUT, "bounded-wait self-test: the wait gave up");
    return CALIB_OK;
}

const char* calib_last_error(void) { return g_err.c_str(); }

void calib_destroy(calib_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    clear_graphs(c);
    free_layout(c);
    for (void* p : {(void*)c->J, (void*)c->Jt, (void*)c->Y, (void*)c->BZ, (void*)c->gradg, (void*)c->grad,
                    (void*)c->x, (void*)c->r, (void*)c->p, (void*)c->Gm,
                    (void*)c->evJ, (void*)c->evE, (void*)c->evOut, (void*)c->part, (void*)c->part_cost, (void*)c->part_dcost,
                    (void*)c->Z, (void*)c->Zprev, (void*)c->basis_d, (void*)c->Pinv_d, (void*)c->freqs_d,
                    (void*)c->rho_d, (void*)c->st, (void*)c->prim, (void*)c->dual2,
                    (void*)c->basis_df, (void*)c->Pinv_df, (void*)c->rinv_df, (void*)c->prim_part, (void*)c->pen_part,
                    (void*)c->rec_part, (void*)c->rec_count, (void*)c->stats, (void*)c->iter_counter,
                    (void*)c->status, (void*)c->part_hv.pn, (void*)c->part_tr.pn, (void*)c->evL, (void*)c->evG, (void*)c->T_d, (void*)c->vis_off_d,
                    (void*)c->coh_off_d, c->staging, (void*)c->ws_prev, (void*)c->ws_mlp, (void*)c->ws_L,
                    (void*)c->xf_d, (void*)c->ws_chose, (void*)c->sgU, (void*)c->sgS, (void*)c->sgJ, (void*)c->sgJt,
                    (void*)c->sgY, (void*)c->sgBZ, (void*)c->sgGradg, (void*)c->sgGrad, (void*)c->sgX, (void*)c->sgR,
                    (void*)c->sgP, (void*)c->sgGm, (void*)c->sgSt})
        if (p) cudaFree(p);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
