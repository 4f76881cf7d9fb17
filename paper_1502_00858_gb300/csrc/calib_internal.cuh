// Internal declarations shared by the CUDA translation units of libcalib.so.
//
// Device data layout (all float32 unless noted; "block" = one 2x2 complex matrix = 8 floats):
//   J, Jt, Y, BZ, gradg, grad, x, r, p   [A][K][N][8]
//   Gm        [A][K][N][4]   Jacobi blocks G_pk (Hermitian): g00, g11, re g01, im g01
//   gw        [A][K][N][NW]  Jacobi weights, rows padded to NW = roundup(N, 4) with zeros:
//                            gw[a][k][p][o] = s_bk = sum_t |c_btk|^2 of the baseline b = (p, o) (symmetric;
//                            0 where flagged or o = p); G_pk = sum_o gw[a][k][p][o] J_ok^H J_ok
//   part      [A][stride][K][N][8]  partial station sums of a baseline sweep (per chunk for the direct
//                                   sweeps, per (agent, CTA) piece for the statistics sweeps)
//   part_cost [A][stride]  float64 partial data cost
//   Z, Zprev  [I][K][M][N][8] float64
//
// Sufficient statistics of a slot (C = c I_2 and J constant over the interval make them exact):
//   U_k = sum_t conj(c_tk) V_t (K 2x2 blocks), S_kl = sum_t conj(c_tk) c_tl (K x K Hermitian, upper
//   triangle packed row-major: entry (k,l), k <= l, at k*K - k*(k-1)/2 + (l-k)).
//
// Baselines are re-laid out per agent by circulant diagonal: diagonal d (1 <= d <= N/2) holds
// the pairs (i, (i+d) mod N); within one diagonal every station is the first element of at most
// one pair and the second element of at most one pair, which makes the per-station reductions
// of the sweeps conflict-free. Data of a pair stored "reversed" (user pair (p,q) held as (q,p))
// is conjugate-transposed (V) / conjugated (c) on ingestion, so kernels never see orientation.
//   V block of (agent, diagonal): [T_a][n_pad][4] float2 (32 B per slot and sample)
//   C block of (agent, diagonal): [T_a][n_pad][K] float2
// The sufficient statistics use the full circulant layout instead (no compaction): diagonal d of
// agent a holds NP = roundup(N, 4) slot positions, position i = the pair (i, (i+d) mod N)
// (i < N, or i < N/2 on the diagonal d = N/2), zero statistics where the baseline is flagged:
//   U[((a*D + d-1)*NP + i)*K*4 ...]  [K][2][2] float2,   S[((a*D + d-1)*NP + i)*KK ...]  packed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

typedef struct calib_mlp calib_mlp;

namespace calib {

constexpr int MAX_N = 256;
constexpr int MAX_K = 16;
constexpr int MAX_M = 16;

// Programmatic dependent launch (the kernel chain of the LM J-update). A kernel launched by
// launch_k with pdl set may start while the preceding kernel in the stream is still running. It
// executes griddep_wait() before it reads anything that kernel writes and before it writes anything
// that kernel reads or writes; the wait returns once the preceding kernel has completed and its
// memory is visible. It calls griddep_launch_dependents() only after its own wait, so a kernel that
// starts early can rely on every kernel before its immediate predecessor having completed. Launched
// without the attribute, both instructions return at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Budget of a bounded in-kernel wait, in SM clock cycles (about one second at 2 GHz).
constexpr long long WAIT_BUDGET_CYCLES = 2000000000LL;

enum StatusBits : int { STATUS_TIMEOUT = 1, STATUS_NONFINITE = 2 };

struct DiagDesc {     // one per (agent, diagonal)
    long long voff;   // float2 offset of the V block
    long long coff;   // float2 offset of the C block
    int slot_off;     // global index of the first slot of this diagonal in the slot arrays
    int n;            // active (unflagged) slots
    int n_pad;        // padded slot count (multiple of 4, >= n)
    int pad_;
};

struct AgentState {   // per-agent scalars
    double L, g;      // augmented Lagrangian and data cost at the current J
    double L_t, g_t;  // at the LM trial point
    double rz;        // PCG r.z (truncated CG: h(r, r))
    double pred;      // predicted decrease of the LM (or trust-region) step
    double mu, nu;    // LM damping
    int cg_stop;      // PCG stopped (r.z <= 0 or p.Ap <= 0); truncated CG: a TCG_STOP_* reason
    int accepted;     // LM steps accepted (cumulative)
    int rejected;     // LM steps rejected (cumulative)
    int pad_;
    // Riemannian trust region (RTR J-update)
    double delta, delta_bar;  // trust-region radius and its cap ||J0||_h
    double r0sq;              // h(r0, r0) of the current truncated CG
    double ee;                // h(eta, eta) of the current truncated-CG iterate
};

// Why a truncated-CG solve stopped (AgentState.cg_stop in the RTR J-update).
enum TcgStop : int { TCG_RUNNING = 0, TCG_BOUNDARY = 1, TCG_CURVATURE = 2, TCG_RESIDUAL = 3 };

// Arguments of a baseline sweep (residual/gradient pass or Gauss-Newton Hessian-vector pass).
struct SweepArgs {
    const float2* V;        // interleaved visibilities (internal layout)
    const float2* C;        // coherencies (internal layout)
    const DiagDesc* desc;   // [A][D]
    const int* slot;        // per slot: first | second << 8
    const int* T;           // [A] samples per agent
    const float* J;         // [A][K][N][8] operating point
    const float* eta;       // [A][K][N][8] direction (Hessian pass) or LM step x (trial pass)
    float* part;            // [A][n_chunks][K][N][8]
    double* part_cost;      // [A][n_chunks] (residual and trial passes)
    double* part_dcost;     // [A][n_chunks] decrease of the data cost (trial pass)
    int* status;            // status bits, set on a timed-out wait
    int A, N, K, D, n_chunks, chunk_diags, TT, slots_max;
};

struct LMArgs {
    // Partials of the preceding sweep: agent a's pieces j < part_n[a] (part_stride for every agent
    // when part_n is NULL) at part[(a * part_stride + j) * K*N*8], part_cost / part_dcost[a * part_stride + j].
    const float* part; const double* part_cost; const double* part_dcost;
    const int* part_n; int part_stride;
    float* J; float* Jt; const float* Y; const float* BZ;
    float* gradg; float* grad; float* x; float* r; float* p;
    float* Gm;
    const float* gw;        // [A][K][N][NW] Jacobi weights, NW = roundup(N, 4)
    AgentState* st;
    const float* rho;       // [K]
    int A, N, K, D;
    double tau;
    int cost_from_decrease;  // trial cost g(J') = g(J) - decrease (statistics sweeps carry no cost)
    int timing;              // autotuner: PCG step runs its whole path and writes no agent state
    int pdl;                 // launch with programmatic dependent launch (griddep_wait below)
};

// Z-update CTAs per (consensus problem, direction) at most: 32 (station, entry) positions each, N <= 128.
constexpr int Z_SLOTS = 32;
// Agents per CTA of the per-iteration record kernel (one warp each).
constexpr int REC_AGENTS = 2;

struct ConsArgs {
    float* J; float* gradg; float* Gm; float* Y; float* BZ;
    double* Z; double* Zprev;
    const double* basis;    // [P][M]
    const double* Pinv;     // [M][M] (sum_i b_i b_i^T)^-1
    const float* rho;       // [K]
    AgentState* st;
    double* prim;           // [A][K] ||J_ik - B_i Z_k|| after k_bz (the iteration's records use prim_part)
    double* dual2;          // [I * G][K][Z_SLOTS] per-CTA shares of ||Z_k^{n+1} - Z_k^n||^2
    const float2* basis_df; // [P][M] the basis as double-float (hi, lo) pairs
    const float2* Pinv_df;  // [G][M][M] Pinv as double-float pairs
    const float2* rinv_df;  // [K] 1 / rho_k as double-float pairs
    float* prim_part;       // [A][K][Z_SLOTS] per-CTA shares of ||J_ik - B_i Z_k||^2
    float* pen_part;        // [A][K][Z_SLOTS] per-CTA shares of Re tr(Y^H D) + rho/2 ||D||^2, D = J - B Z
    double* rec_part;       // [ceil(A / REC_AGENTS)][3] per-CTA sums of the record kernel
    int* rec_count;         // record-kernel CTAs done in the current launch (0 between launches)
    double* stats;          // [max_iters][4]
    int* iter_counter;
    // Consensus problems: each of the I intervals' P frequencies splits into G interleaved groups
    // (group g = frequency indices g, g + G, ...; G = 1: one problem per interval), each its own
    // C-ADMM problem of P / G agents (frequency multiplexing, Section 3). Problem pb = iv * G + g;
    // its j-th agent is iv * P + g + G * j. Z and Zprev are [I * G][K][M][N][8]; Pinv is [G][M][M].
    int A, I, P, M, N, K, max_iters, G;
};

// ---- launchers (sweep.cu)
enum SweepMode : int { SWEEP_RESIDUAL = 0, SWEEP_HESSVEC = 1, SWEEP_TRIAL = 2 };
cudaError_t launch_sweep(const SweepArgs& a, int mode, cudaStream_t s);
size_t sweep_smem_bytes(int N, int K, bool two_vectors);
int sweep_tile_samples(int slots_max, int K, bool hessvec);
int sweep_threads(int slots_max);

// ---- launchers (lm.cu)
// LM_BEGIN_FROM_TRIAL (trust region only): the gradient comes from the partials of a statistics
// trial pass run at J' = J, which carries no absolute cost (the SAGE sub-problems use decreases only).
enum LMEvalMode : int { LM_BEGIN_FROM_PARTIALS = 0, LM_BEGIN_REUSE = 1, LM_ACCEPT = 2, LM_BEGIN_FROM_TRIAL = 3 };
cudaError_t launch_lm_eval(const LMArgs& a, int mode, cudaStream_t s);
// One PCG step; with last set it also forms the LM trial point Jt = J + x and the predicted decrease.
cudaError_t launch_cg_step(const LMArgs& a, bool last, cudaStream_t s);
cudaError_t launch_eval_output(const LMArgs& a, float* grad_out, double* L_out, double* g_out, cudaStream_t s);
// Riemannian trust-region J-update (the paper's inner solver): one truncated-CG step after the
// Hessian sweep of its direction d (with last set it also forms J' = J + eta and the predicted
// decrease), and the trust-region bookkeeping after a residual or trial sweep (modes in LMEvalMode).
cudaError_t launch_tcg_step(const LMArgs& a, bool last, cudaStream_t s);
cudaError_t launch_rtr_eval(const LMArgs& a, int mode, cudaStream_t s);
cudaError_t launch_hv_output(const LMArgs& a, float* out, cudaStream_t s);

// ---- launchers (sage.cu): the SAGE decomposition of the J-update over directions (step D1)
struct SageArgs {
    const float2* U; const float2* S;       // statistics of all directions (full circulant layout)
    const float* J; const float* Y; const float* BZ;  // [A][K][N][8]
    float* J_out;                           // where direction k's solution is scattered back (= J)
    float2* U1; float2* S1;                 // direction k's one-direction statistics
    float *J1, *Jt1, *Y1, *BZ1;             // [A][N][8] copies of direction k's vectors
    int A, D, NP, K, N;
};
cudaError_t launch_sage_prepare(const SageArgs& g, int k, cudaStream_t s);
cudaError_t launch_sage_scatter(const SageArgs& g, int k, cudaStream_t s);

// ---- launchers (consensus.cu)
cudaError_t launch_gauge(const ConsArgs& a, cudaStream_t s);
// Z-update (Eq. Zest) and Y-update (Eq. M3) of one C-ADMM iteration in one launch, then the
// iteration's records (Section 4) and each agent's L_i.
cudaError_t launch_zy_update(const ConsArgs& a, cudaStream_t s);
cudaError_t launch_records(const ConsArgs& a, cudaStream_t s);
cudaError_t launch_bz_only(const ConsArgs& a, cudaStream_t s);
cudaError_t launch_identity(float* J, long long n_blocks, cudaStream_t s);

// ---- launchers (data.cu)
struct IngestArgs {
    const float2* src;          // user layout [A][B][T_a][w] (w = 4 for V, K for C)
    const long long* src_off;   // [A] float2 offset of each agent's [B][T_a][w] block
    const uint8_t* flags;       // unused here (slots already compacted)
    float2* dst;
    const DiagDesc* desc; const int* slot; const int* slot_b; const int* T;
    int A, D, K, is_vis;
};
cudaError_t launch_ingest(const IngestArgs& a, cudaStream_t s);
cudaError_t launch_extract_coh(const IngestArgs& a, float2* user_dst, cudaStream_t s);
struct ResidualArgs {
    const float2* V; const float2* C;  // internal layouts
    const float* J;                    // [A][K][N][2][2] complex
    float2* out;                       // user layout [A][B][T_a][2][2]
    const long long* vis_off;          // [A] float2 offset of each agent's block in out
    const DiagDesc* desc; const int* slot; const int* slot_b; const int* T;
    int A, D, K, N;
    unsigned mask;                     // bit k: subtract direction k's model
    int correct;                       // direction whose solutions correct the residual, -1: none
};
cudaError_t launch_residual(const ResidualArgs& a, cudaStream_t s);
struct PredictArgs {
    const double* uvw;      // [I][Tmax][N][3]
    const double* sky;      // [K][S][4]
    const double* freqs;    // [P]
    double f0;
    float2* C;
    const DiagDesc* desc; const int* slot; const int* T;
    int A, P, N, K, S, D, Tmax;
};
cudaError_t launch_predict(const PredictArgs& a, cudaStream_t s);
cudaError_t launch_gram_weights(const float2* C, const DiagDesc* desc, const int* slot, const int* T, float* gw,
                                int A, int D, int K, int N, cudaStream_t s);
cudaError_t launch_check_finite(const float* x, long long n, int* status, cudaStream_t s);
// Statistics into the full circulant layout (positions of flagged baselines are not written).
cudaError_t launch_ss_stats(const float2* V, const float2* C, float2* U, float2* S, const DiagDesc* desc,
                            const int* slot, const int* T, int A, int D, int K, int N, int Tmax, int* status,
                            cudaStream_t s);

// ---- launchers (ss.cu): sweeps on the sufficient statistics
struct SSArgs {
    const float2* U; const float2* S;    // full circulant layout, NP positions per diagonal
    const float* J; const float* eta;   // eta: direction (Hessian) or LM step x (trial)
    float* part; double* part_dcost; int* status;
    int A, N, K, D, NP;
    int part_stride;   // pieces per agent in part / part_dcost (>= the CTAs meeting any one agent)
    int pdl;           // launch with programmatic dependent launch; the statistics must not be
                       // written by the preceding kernel (they are read before griddep_wait)
};
// grid CTAs split the A*D (agent, diagonal) items into equal contiguous ranges; 1 <= grid <= A*D.
cudaError_t launch_ss_sweep(const SSArgs& a, bool hessvec, int grid, cudaStream_t s);
size_t ss_sweep_smem_bytes(int N, int K, bool hessvec, int* stage_bytes);
int ss_sweep_threads(int N);
cudaError_t prepare_ss_kernels();
// the one-thread-per-slot Hessian pass (K <= 5, ss_hessvec.cu)
cudaError_t prepare_ss_hessvec_kernels();
cudaError_t launch_ss_hessvec1(const SSArgs& a, int grid, int threads, size_t smem, int sb, cudaStream_t s);

// One-time kernel attribute set-up (dynamic shared memory limits); call before any capture.
cudaError_t prepare_sweep_kernels();
cudaError_t prepare_lm_kernels();
cudaError_t prepare_data_kernels();

// Warm-start network pieces (mlp.cu) used by calib_warm_start.
cudaError_t mlp_warm_rows(calib_mlp* h, const float* J_prev, const float* BZ, const double* xf, int K, int N, int A,
                          float* J_mlp, cudaStream_t s);
cudaError_t mlp_warm_select(const float* J_mlp, const float* J_prev, const double* L_mlp, const double* L_prev, int KN8,
                            int A, float* J_out, int* chose, cudaStream_t s);
cudaError_t launch_ws_features(const float* J, const float* BZ, const double* xf, int K, int N, long long rows, float* X,
                               cudaStream_t s);

// Record the message returned by calib_last_error() on this thread (capi.cu).
void set_last_error(const std::string& msg);

}  // namespace calib
