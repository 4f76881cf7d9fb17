/*
 * calib.h - C ABI of the GB300 consensus-ADMM calibration library (libcalib.so).
 *
 * The library runs distributed (consensus) radio-interferometric calibration across
 * frequency, Yatawatta 2015 (arXiv:1502.00858), on one GPU. The paper's P compute
 * agents - one per frequency f_i - become slices of single kernel launches; several
 * independent solution intervals (the paper calibrates every 200 s of data
 * separately, Section 4) are batched the same way. One call of calib_admm_iter runs
 * C-ADMM iterations (Section 3, Eq. M1-M3, steps D1-D3):
 *
 *   M1  J_i <- argmin_J L_i(J, Z, Y_i)       per agent, by Levenberg-Marquardt with
 *                                            preconditioned CG steps (default), or by the
 *                                            paper's RTR or SAGE (calib_options.jupdate)
 *   M2  Z   <- closed form of Eq. Zest        per interval and direction (fusion centre)
 *   M3  Y_i <- Y_i + rho (J_i - B_i Z)        per agent
 *
 * J and Y are float32; Z is stored in float64 and M2/M3 are computed in double-float
 * arithmetic (pairs of float32, about 48 bits). Every reduction runs in a fixed order, so a
 * call repeats bit for bit (calib_eval_noalloc, whose sums use atomics, excepted).
 *
 * with L_i(J,Z,Y) = g(J) + Re tr(Y^H (J - B Z)) + rho/2 ||J - B Z||^2 (Eq. sumtrace2),
 * g(J) = sum_t sum_{p<q} ||V_pq - sum_k J_pk C_pqk J_qk^H||^2 (Eq. mltheta / Eq. sum3)
 * and C_pqk = c_pqk I_2 for unpolarised sources (Eq. coh).
 *
 * Symbols: N stations, B baselines (pairs p<q), K directions, P frequencies (agents
 * per interval), M basis terms (the paper calls this F), I solution intervals,
 * A = I*P agents (agent a = interval*P + frequency index), T_a samples of agent a,
 * G frequency groups per interval (calib_options.freq_groups, default 1): I*G consensus
 * problems, problem (interval, g) holding the agents of frequency indices g, g+G, ...
 *
 * Conventions for every entry point:
 *  - Return value: CALIB_OK (0) or a negative CALIB_E* code; calib_last_error() then
 *    holds a message for the calling thread. No C++ exception or abort crosses the ABI.
 *  - Complex arrays are interleaved (re, im) float32 ("c64") unless stated as c128.
 *  - ptr_kind 0: host pointers. The call copies inputs before returning and writes
 *    outputs before returning (it synchronises the library stream).
 *    ptr_kind 1: device pointers, ordered on the library stream (calib_options.cuda_stream).
 *    Device inputs must stay valid until the stream reaches the call; device outputs are
 *    complete once the stream passes the call (calib_sync waits for it).
 *  - The context owns all of its device memory and frees it in calib_destroy.
 *  - A context is not thread-safe: one thread at a time per context.
 */
#ifndef CALIB_H
#define CALIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CALIB_OK = 0,
    CALIB_EINVAL = -1,   /* bad argument: size, index, layout, non-positive rho, ... */
    CALIB_ERANK = -2,    /* P < M or sum_i b_i b_i^T singular (Section 3, "P >= F") */
    CALIB_ENOMEM = -3,   /* device or host allocation failed */
    CALIB_ECUDA = -4,    /* a CUDA runtime call failed (message names it) */
    CALIB_ETIMEOUT = -5, /* a bounded wait inside a kernel gave up; results are invalid */
    CALIB_ENUMERIC = -6, /* non-finite input data */
    CALIB_ESTATE = -7    /* call order: e.g. calib_admm_iter before any data was set */
};

typedef struct calib_ctx calib_ctx;

/* How the LM/PCG passes of the J-update read the data (calib_options.formulation). Both compute
 * the same quantities (the sums over the samples of a baseline, Section 2):
 *  CALIB_FORM_STATISTICS  per-baseline sufficient statistics U_k = sum_t conj(c_tk) V_t and
 *                         S_kl = sum_t conj(c_tk) c_tl, formed once per data set (exact because
 *                         C = c I_2 and J is constant over an interval); passes no longer depend on T;
 *  CALIB_FORM_DIRECT      every pass streams the visibilities and coherencies sample by sample. */
enum { CALIB_FORM_STATISTICS = 0, CALIB_FORM_DIRECT = 1 };

/* The inner solver of the J-update (calib_options.jupdate), Eq. M1:
 *  CALIB_JUPDATE_LM   n_lm Levenberg-Marquardt steps, each with n_cg preconditioned CG steps on the
 *                     damped Gauss-Newton system (block-Jacobi preconditioner, Nielsen damping);
 *  CALIB_JUPDATE_RTR  the paper's Riemannian trust-region method (Section 3, Appendix A) in
 *                     Euclidean space (retraction J + eta): n_lm trust-region steps, each with up to
 *                     n_cg truncated-CG steps (Steihaug-Toint, unpreconditioned, norm sqrt(h(x, x)),
 *                     stopping on the boundary, on non-positive curvature or when
 *                     ||r|| <= ||r0|| min(||r0||, 0.1)); step accepted when the ratio of actual to
 *                     model decrease exceeds 0.1; radius quartered below 1/4, doubled (capped at
 *                     ||J0||_h) above 3/4 when the CG stopped on the boundary; initial radius
 *                     ||J0||_h / 8 at the start of every J-update;
 *  CALIB_JUPDATE_SAGE the SAGE decomposition over directions (step D1): n_sage sweeps, each
 *                     visiting k = 0 .. K-1; direction k's expectation step removes the other
 *                     directions' models from the data (done exactly on the per-baseline statistics:
 *                     U_k - sum_{l != k} S_kl J_pl J_ql^H, S_kk), and its maximisation step is the RTR
 *                     above (n_lm steps of up to n_cg truncated-CG steps) on direction k's own
 *                     Lagrangian with full regularisation. Needs CALIB_FORM_STATISTICS. */
enum { CALIB_JUPDATE_LM = 0, CALIB_JUPDATE_RTR = 1, CALIB_JUPDATE_SAGE = 2 };

typedef struct {
    int n_intervals;                   /* I >= 1 (default 1) */
    int n_samples;                     /* T >= 1: samples per agent when samples_per_agent is NULL */
    const int32_t* samples_per_agent;  /* [A] samples of each agent, or NULL (host pointer, copied) */
    int n_lm;                          /* LM (or trust-region) steps per J-update (default 10) */
    int n_cg;                          /* PCG (or truncated-CG) steps per LM step (default 4) */
    int chunk_diagonals;               /* direct sweeps: baseline diagonals per CTA; 0 = automatic */
    void* cuda_stream;                 /* cudaStream_t to run on; NULL = the library creates one */
    int formulation;                   /* CALIB_FORM_STATISTICS (default) or CALIB_FORM_DIRECT */
    int ctas_per_sm;                   /* statistics sweeps: grid = SMs * ctas_per_sm CTAs (at most one
                                          per agent-diagonal), each taking an equal contiguous share of
                                          the (agent, diagonal) items; 0 = automatic */
    int jupdate;                       /* CALIB_JUPDATE_LM (default), CALIB_JUPDATE_RTR or CALIB_JUPDATE_SAGE */
    int n_sage;                        /* SAGE sweeps per J-update (default 1; CALIB_JUPDATE_SAGE only) */
    int freq_groups;                   /* G >= 1 (default 1; 0 is taken as 1), dividing P: frequency multiplexing. With more
                                          frequencies than agents per consensus problem (Section 3), each
                                          interval's P frequencies form G interleaved subsets - subset g is
                                          the frequency indices g, g+G, g+2G, ... (each spans the band) -
                                          and every subset is its own C-ADMM problem of P/G agents with its
                                          own Z (the paper repeats the selection sequentially; here the
                                          I*G problems run in the same batch). Needs P/G >= M. */
} calib_options;

/* One record per C-ADMM iteration (Section 4 definitions, summed/averaged over all intervals):
 *  primal     mean over agents i and directions k of ||J_ik - B_i Z_k|| / sqrt(4N)
 *  dual       mean over intervals and directions of ||Z_k^{n+1} - Z_k^n|| / sqrt(4MN)
 *  objective  sum_i L_i(J_i^{n+1}, Z^{n+1}, Y_i^{n+1})
 *  resid_norm sqrt(sum_i g_i(J_i^{n+1}))                                              */
typedef struct {
    double primal;
    double dual;
    double objective;
    double resid_norm;
} calib_stats;

/* Fill *opt with the defaults listed above. */
void calib_default_options(calib_options* opt);

/* Create a context for a fixed problem shape (Section 3 problem statement, Eq. hidden,
 * Eq. poly, Eq. Zest).
 *  n_stations N in [2, 128]; n_baselines B in [1, N(N-1)/2];
 *  pq        [B][2] int32 station pairs with 0 <= p < q < N, no duplicates (host);
 *  n_dirs    K in [1, 16];   n_freqs P >= 1;   freqs_hz [P] (host; stored for calib_predict);
 *  n_basis   M in [1, 16] with P >= M;  basis [P][M] row-major b_l(f_i) (host, float64);
 *  rho       [K] per-direction regularisation, each > 0 (Section 3) (host);
 *  opt       may be NULL (defaults).
 * Computes (sum_i b_i b_i^T)^-1 in float64; returns CALIB_ERANK when it does not exist.
 * The state starts cold: J = identity blocks, Z = Y = 0 (Section 3, initialisation). */
int calib_init(calib_ctx** out, int n_stations, int n_baselines, const int32_t* pq,
               int n_dirs, int n_freqs, const double* freqs_hz, int n_basis,
               const double* basis, const double* rho, const calib_options* opt);

/* Load observed data (Eq. vispq).
 *  vis   c64, agent-major packed [A][B][T_a][2][2] (the 2x2 block row-major: XX XY YX YY);
 *  coh   c64 [A][B][T_a][K] scalar coherencies c with C = c I_2, or NULL when calib_predict
 *        will supply them;
 *  flags uint8 [A][B], 1 = exclude this baseline of this agent from g (host or device per
 *        ptr_kind), or NULL = nothing flagged. Flags are fixed at the first call.
 * Rejects non-finite visibilities or coherencies (CALIB_ENUMERIC) when ptr_kind is 0; the
 * context then holds no data (and no coherencies, if coh was given) until a call succeeds. */
int calib_set_data(calib_ctx* ctx, const void* vis, const void* coh, const uint8_t* flags, int ptr_kind);

/* Predict the scalar coherencies of point-source clusters (Eq. coh) on the GPU.
 *  uvw_m  float64 [I][Tmax][N][3] per-station (u,v,w) in metres (agent a uses the first T_a
 *         samples of its interval);  Tmax = max_a T_a;
 *  sky    float64 [K][S][4] per cluster: l, m (direction cosines), I0 (flux at f0_hz), alpha;
 *  f0_hz  reference frequency of the spectral indices.
 * Phase reading: c_pq = sum_s I0_s (f/f0)^alpha_s exp(i phi), phi = -2 pi (f/c)
 * (u_pq l + v_pq m + w_pq (sqrt(1-l^2-m^2)-1)), (u,v,w)_pq = (u,v,w)_p - (u,v,w)_q.
 * Turns are formed in float64 per station and reduced to [-1/2, 1/2) before float32
 * sincospi. Replaces any coherencies given to calib_set_data. */
int calib_predict(calib_ctx* ctx, const double* uvw_m, const double* sky, int n_src,
                  double f0_hz, int ptr_kind);

/* Copy the coherencies in use out in the calib_set_data layout [A][B][T_a][K] c64
 * (flagged baselines read as 0). */
int calib_get_coherencies(calib_ctx* ctx, void* coh, int ptr_kind);

/* Cold start: J = identity blocks, Z = Y = 0; the next iteration applies the first-iteration
 * gauge projection (Section 3, initialisation). */
int calib_reset(calib_ctx* ctx);

/* Set J (c64 [A][K][N][2][2]) as the starting point of the next J-update, for a warm start
 * from a previous solution interval (Section 3, initialisation). Z and Y are unchanged. */
int calib_set_initial(calib_ctx* ctx, const void* J0, int ptr_kind);

/* Set the consensus state: Z c128 [I][G][K][M][N][2][2] and Y c64 [A][K][N][2][2] (either may
 * be NULL = zero). B_i Z is recomputed. A state set this way is warm: no gauge projection.
 * With calib_get_solutions this is checkpoint and resume. */
int calib_set_consensus(calib_ctx* ctx, const void* Z, const void* Y, int ptr_kind);

/* Run n_iters C-ADMM iterations (Eq. M1-M3). If hist is not NULL it receives n_iters
 * records (host memory, written before return). Returns CALIB_ETIMEOUT if a bounded
 * in-kernel wait gave up. */
int calib_admm_iter(calib_ctx* ctx, int n_iters, calib_stats* hist);

/* Copy out J c64 [A][K][N][2][2], Z c128 [I][G][K][M][N][2][2], Y c64 [A][K][N][2][2].
 * Any pointer may be NULL. */
int calib_get_solutions(calib_ctx* ctx, void* J, void* Z, void* Y, int ptr_kind);

/* Checkpoint and resume of the iteration state (the paper restarts a calibration from the
 * previous time slot's solutions, Section 3, initialisation; this keeps the whole C-ADMM state).
 * The blob is opaque, host memory, and holds J, Y, B_i Z, Z, Z^{n-1}, the projected data gradient
 * and Jacobi blocks at J, the per-agent LM scalars (L, g, damping), the pending first-iteration
 * gauge-projection flag and the number of iterations since the last cold start; the data
 * (visibilities, coherencies, flags) are not in it. After calib_set_state the next
 * calib_admm_iter continues exactly (bit for bit) where the saved context stood.
 *  calib_get_state: buf NULL -> *len receives the size needed; else *len is the buffer's size
 *    (CALIB_EINVAL, with the size needed in *len, if too small) and receives the bytes written.
 *    Synchronises the context's stream.
 *  calib_set_state: CALIB_EINVAL if the blob is not one, or was saved for another shape,
 *    formulation, station-pair list, sample counts or flags. Synchronises the stream. */
int calib_get_state(calib_ctx* ctx, void* buf, size_t* len);
int calib_set_state(calib_ctx* ctx, const void* buf, size_t len);

/* Per-agent L_i and g_i after the last iteration, float64 [A] each (host). Either may be NULL. */
int calib_get_agent_objective(calib_ctx* ctx, double* L, double* g);

/* Evaluate the augmented Lagrangian and its gradient at a given J (c64 [A][K][N][2][2])
 * with the context's current Z and Y: L float64 [A], g float64 [A] (either may be NULL),
 * grad c64 [A][K][N][2][2] = grad_i(L_i, J) of Eq. gradL (gradient w.r.t. the inner
 * product h of Eq. inprod; the real-coordinate gradient is twice this). Does not change
 * the iteration state. L and g are host arrays when ptr_kind is 0, else device. */
int calib_eval(calib_ctx* ctx, const void* J, double* L, double* g, void* grad, int ptr_kind);

/* Gauss-Newton Hessian-vector product of L_i at J along eta (Eq. HessL with the GN part of
 * Hess g): out c64 [A][K][N][2][2]. Inputs and output as in calib_eval. */
int calib_hessvec(calib_ctx* ctx, const void* J, const void* eta, void* out, int ptr_kind);

/* Wait until all work queued on the library stream has finished. */
int calib_sync(calib_ctx* ctx);

/* Per-kernel timing over the following calib_admm_iter calls (CUDA events recorded
 * on the library stream around every launch of the sweep and per-agent LM kernels when enabled).
 * Kinds: sweep_residual (direct residual/trial), sweep_hessvec (direct Hessian), stats_hessvec and
 * stats_trial (sufficient-statistics passes), pcg_step and lm_eval (per-agent LM kernels, no
 * algorithmic byte or flop count: 0), stats_pass (forming the statistics from V and C, timed
 * outside the graph when calib_admm_iter runs it), consensus (the gauge projection, Z-update,
 * Y-update and records of one iteration, timed as one); bytes_per_launch and flops_per_launch are the
 * algorithmic bytes and real flops (complex multiply 6, complex multiply-add 8) of one launch.
 * Every output array may be NULL and receives up to cap entries; returns the number of kinds. */
int calib_profile_enable(calib_ctx* ctx, int on);
int calib_profile_read(calib_ctx* ctx, int cap, const char** names, double* total_ms,
                       long long* launches, double* bytes_per_launch, double* flops_per_launch);

/* Autotuner: time the two halves of one LM step on the loaded data - n_cg Hessian passes with
 * their PCG steps, and the trial pass with its reduction - for each candidate work split. The
 * split is CTAs per SM (1, 2, 3, 4, 5, 6, 8, 12, 16, 24) for CALIB_FORM_STATISTICS, chosen per pass,
 * and diagonals per CTA (1, 2, 4, ..., N/2) for CALIB_FORM_DIRECT, one value for both passes (the
 * fastest whole step). calib_admm_iter runs it by itself before its first iteration when the
 * option that fixes the split (ctas_per_sm or chunk_diagonals) is 0; the choice is cached per
 * problem shape for the process. This call re-measures. Outputs (host, any may be NULL): the
 * chosen split of the Hessian and of the trial pass, up to cap candidates with the milliseconds of
 * each half, and the candidate count. The iteration state (J, Z, Y) is not changed. */
int calib_autotune(calib_ctx* ctx, int* split, int* split_trial, int cap, int* candidates,
                   double* ms_hessian, double* ms_trial, int* n_candidates);

/* ---- Learned warm start (the paper starts a calibration from the previous time slot's solution,
 * Section 3, initialisation; a small network refines that start).
 * Network: rows of 17 inputs (J_prev of one station and direction as 8 reals (re, im of the 2x2
 * row-major entries), (B_f Z_prev) likewise, normalised frequency (f - f_min)/(f_max - f_min)),
 * `depth` ReLU layers of `width`, 8 outputs y; J_init = J_prev + y. bfloat16 weights and biases
 * (copies of float32 master weights), float32 accumulation; AdamW on the mean squared error.
 * Weights are a flat float32 array [W_1 (width x 17), b_1, ..., W_last (8 x width), b_last],
 * row-major; calib_mlp_num_params gives its length. A network has its own stream (cuda_stream
 * NULL = its own) and is not thread-safe. The paper has no network: it refines the paper's
 * previous-solution start, and its output is kept only where the ADMM's own objective
 * accepts it (calib_warm_start). */
typedef struct calib_mlp calib_mlp;
int calib_mlp_create(calib_mlp** out, int n_in, int width, int depth, int n_out, void* cuda_stream);
long long calib_mlp_num_params(calib_mlp* mlp);
int calib_mlp_set_weights(calib_mlp* mlp, const float* w, int ptr_kind);   /* resets the optimiser */
int calib_mlp_get_weights(calib_mlp* mlp, float* w, int ptr_kind);
/* y [rows][8] for rows X [rows][17] (float32). */
int calib_mlp_forward(calib_mlp* mlp, const float* X, float* Y, int rows, int ptr_kind);
/* Loss mean_r ||X[r,0:8] + y_r - T_r||^2 and its gradient w.r.t. the float32 weights (flat layout);
 * grad and loss may be NULL. */
int calib_mlp_grad(calib_mlp* mlp, const float* X, const float* T, int rows, float* grad, double* loss, int ptr_kind);
/* One AdamW step (beta 0.9/0.999, eps 1e-8, decoupled weight decay) on a batch; loss before the step. */
int calib_mlp_train_step(calib_mlp* mlp, const float* X, const float* T, int rows, float lr, float weight_decay,
                         double* loss, int ptr_kind);
void calib_mlp_destroy(calib_mlp* mlp);
/* Feature rows [A*K*N][17] of the context's current state (J and B_f Z after the last iteration,
 * normalised frequency), rows ordered (agent, direction, station): the network's inputs for the
 * following interval. */
int calib_get_features(calib_ctx* ctx, float* X, int ptr_kind);
/* Warm start of the next calib_admm_iter from the previous interval's solution J_prev c64 [A][K][N][2][2]
 * and consensus Z_prev c128 [I][G][K][M][N][2][2]: Z = Z_prev, Y = 0 (warm: no gauge projection), and per
 * agent J = J_prev + network(J_prev, B_f Z_prev, f) where that gives the lower L_i, else J = J_prev
 * (mlp NULL: always J_prev). chose [A] (may be NULL) receives 1 where the network's start was kept. */
int calib_warm_start(calib_ctx* ctx, calib_mlp* mlp, const void* J_prev, const void* Z_prev, int* chose, int ptr_kind);

/* Residual visibilities after calibration (Section 2: the solutions correct the data, and the
 * residual is the data minus the predicted model), from the context's visibilities, coherencies and
 * current solutions J (after calib_admm_iter, calib_set_initial or calib_warm_start):
 *    R_pq = V_pq - sum_{k : subtract[k] != 0} J_pk C_pqk J_qk^H,
 * then, if correct_dir >= 0, R_pq <- J_p,c^-1 R_pq J_q,c^-H with c = correct_dir (the data corrected
 * for that direction's errors; correcting first and subtracting the corrected model is the same).
 *  subtract: host int32 [K], nonzero = subtract direction k's model; NULL = every direction.
 *  out: c64 [A][B][T_a][2][2], the layout of calib_set_data's visibilities; host (ptr_kind 0,
 *       written before return) or device (ptr_kind 1, stream-ordered on the context's stream).
 *       Flagged baselines are written as zeros. A singular J_p,c gives non-finite values there.
 * Returns CALIB_ESTATE before visibilities and coherencies are set, CALIB_EINVAL for correct_dir
 * outside [-1, K). */
int calib_residual(calib_ctx* ctx, const int32_t* subtract, int correct_dir, void* out, int ptr_kind);

/* Number of kernels this context has launched since creation (all kinds). */
long long calib_launch_count(calib_ctx* ctx);

/* Size in bytes of the fixed device array that calib_eval_noalloc uses as scratch. */
#define CALIB_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)

/* calib_eval without any allocation, for callers that cannot call cudaMalloc: applications
 * whose device memory is all reserved by their own pool allocator (a cudaMalloc would fail or
 * fragment it), and latency-critical pipelines that cannot take the implicit device
 * synchronisation of cudaMalloc / cudaFree. The paper has no counterpart; it is a deployment
 * variant of the residual/gradient evaluation.
 *  Inputs (device pointers, read in order on cuda_stream; NULL stream = legacy default):
 *    pq int32 [B][2] with 0 <= p < q < N, checked on the device: a pair outside that range is
 *       skipped and every agent's L, g and grad are written as NaN (the call itself returns
 *       CALIB_OK, since it does not wait for the GPU);
 *    vis c64 [A][B][T][2][2]; coh c64 [A][B][T][K];
 *    J c64 [A][K][N][2][2]; Y and BZ c64 [A][K][N][2][2] (either NULL = zero); rho host float64 [K].
 *    Every agent uses all B baselines and T samples (no flags).
 *  Outputs (device): L and g float64 [A] (either NULL = not written), grad c64 [A][K][N][2][2]
 *    = grad_i(L_i, J) of Eq. gradL; the same quantities as calib_eval.
 * Scratch: per-chunk partial sums live in one static device array of CALIB_NOALLOC_SCRATCH_BYTES
 * (8 MiB), held by every GPU that loads the library until the process exits. A problem needing
 * more, A * ceil(B/256) * (32 K N + 8) bytes, is rejected with CALIB_EINVAL. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture. All calls share the array and it keeps the
 * last call's contents (each call rewrites what it reads, so nothing needs clearing); calls that
 * overlap on the GPU race on it and must be serialised by the caller. The station sums are
 * accumulated with shared-memory atomics in no fixed order, so, unlike calib_eval, results are
 * not bitwise reproducible from call to call (they agree to float32 rounding). Returns after
 * enqueueing (asynchronous); errors of the launch are reported, errors of execution surface at
 * the next synchronisation. */
int calib_eval_noalloc(int n_agents, int n_stations, int n_baselines, int n_dirs, int n_samples,
                       const int32_t* pq, const void* vis, const void* coh, const void* J,
                       const void* Y, const void* BZ, const double* rho, double* L, double* g,
                       void* grad, void* cuda_stream);

/* Self-test of the failure path shared by every kernel that waits on its own bulk copies: one
 * CTA waits, with the library's bounded wait (about one second of SM clock), on an mbarrier
 * phase. complete_phase != 0 completes the phase before the wait (control: returns CALIB_OK);
 * complete_phase == 0 leaves it pending, so the wait gives up, the kernel records a timeout in
 * a status word and returns, and the call returns CALIB_ETIMEOUT with the context of the device
 * still usable. No copy is issued, so nothing is in flight when the wait gives up. The paper has
 * no counterpart. cuda_stream as in calib_options (NULL = legacy default); the call allocates a
 * 4-byte status word, synchronises the stream, and writes the kernel's duration in milliseconds
 * (CUDA events) to elapsed_ms (may be NULL). CALIB_ECUDA if a CUDA call fails. */
int calib_selftest_bounded_wait(int complete_phase, double* elapsed_ms, void* cuda_stream);

/* Message of the last failing call on this thread ("" if none). */
const char* calib_last_error(void);

/* Free the context and all device memory it owns. NULL is allowed. */
void calib_destroy(calib_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* CALIB_H */
