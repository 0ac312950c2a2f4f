/*
 * tns.h -- C ABI of the GB300 boundary-MPS sampler for 2D tensor-network states.
 *
 * Method: Rudolph & Tindall, "Simulating and Sampling from Quantum Circuits with
 * 2D Tensor Networks" (arXiv 2507.11424).  A processor-shaped tensor-network
 * state (one tensor per qubit, bonds on the coupling graph; Methods) is built by
 * belief-propagation-gauged simple update (Methods, Eqs. 1-2; Appendix Fig. 8)
 * and sampled with the generalized boundary-MPS contraction (Appendix,
 * "Sampling from a Tensor Network State", Fig. 7).
 *
 * Conventions shared by every entry point:
 *   - All functions return a tns_status; no exception crosses the ABI.  After
 *     any error other than TNS_ERR_CUDA the state stays valid.  A thread-local
 *     message is available from tns_last_error().
 *   - Host arrays passed in are read during the call only (the caller keeps
 *     ownership).  Device buffers passed in are caller-owned device memory on the
 *     device that was current when the state was created; they are accessed on
 *     the state's stream, and the call returns once that stream has finished
 *     using them.
 *   - Complex numbers are interleaved (re, im) float64 pairs.
 *   - Qubit indices are the positions in the arrays given to tns_build_lattice;
 *     bit x_q = 1 means |1>.
 *   - A state is used by one host thread at a time.
 */
#ifndef TNS_H
#define TNS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TNS_OK = 0,
  TNS_ERR_ARG = 1,            /* invalid argument (sizes, indices, non-disjoint gates, ...) */
  TNS_ERR_CUDA = 2,           /* a CUDA call failed; the state must be destroyed */
  TNS_ERR_OOM = 3,            /* device allocation failed */
  TNS_ERR_NOT_CONVERGED = 4,  /* BP stopped at max_iter; outputs hold the last iterate */
  TNS_ERR_NUMERIC = 5,        /* NaN/Inf met, or a Jacobi sweep cap was reached */
  TNS_ERR_STATE = 6           /* call not valid for this state (e.g. wrong file format) */
} tns_status;

typedef enum {
  TNS_PREC_FP64 = 0,  /* every contraction and factorisation in FP64 */
  TNS_PREC_MIXED = 1  /* complex64 storage; contractions on the tensor cores as a TF32
                         three-pass split (FP32-level accuracy) or on FP32 CUDA cores;
                         truncation Grams, Cholesky and Jacobi in FP32; probabilities and
                         log q in FP64 */
} tns_prec;

typedef struct tns_state tns_state; /* opaque, library-owned */

/*
 * tns_build_lattice -- processor-shaped product state (Methods, first paragraph:
 * one tensor per qubit, virtual bonds on the coupling graph).
 *   n_sites   number of qubits (>= 1)
 *   grid_rc   host int32 [n_sites][2]: (row, col) grid cell of each qubit; cells
 *             must be distinct and non-negative.  The grid is transposed inside
 *             the library when it has more columns than rows, so that the
 *             boundary MPS runs along the shorter side.
 *   n_edges, edges  host int32 [n_edges][2]: bonded qubit pairs; each pair must
 *             occupy nearest-neighbour grid cells (planar grid embedding).
 *   init_bits host uint8 [n_sites]: initial computational basis state.
 *   chi_max   largest bond dimension any later call may request (sizes storage).
 *   prec      default precision of tns_sample / tns_amplitude.
 *   cuda_stream  cudaStream_t to run on (NULL = legacy default stream).
 *   out       receives the new state (NULL on failure).
 * Every bond starts at dimension 1 and every BP message at [1].
 */
tns_status tns_build_lattice(int32_t n_sites, const int32_t* grid_rc, int32_t n_edges, const int32_t* edges,
                             const uint8_t* init_bits, int32_t chi_max, tns_prec prec, void* cuda_stream,
                             tns_state** out);

/*
 * tns_apply_gate_layer -- apply one group of non-overlapping gates (Methods,
 * edge colouring; Eq. HeisenbergProp) by BP-gauged simple update (Appendix,
 * "Applying Gates", Fig. 8d): gauge each gate's two sites with the square roots
 * of their incoming BP messages, reduce to R factors by QR, apply the gate,
 * truncate the SVD to chi (Eq. 1), ungauge.  One-qubit gates are contracted
 * exactly.  The state is not renormalised.
 *   n_gates   number of gates; their qubits must be pairwise distinct
 *   sites     host int32 [n_gates][2]; sites[g][1] = -1 marks a one-qubit gate;
 *             two-qubit gates must act on a bonded pair
 *   mats      host float64 [n_gates][16][2]: complex matrix, row-major,
 *             U[2*o0 + o1][2*i0 + i1] with qubit sites[g][0] the high bit; a
 *             one-qubit gate uses the first 4 entries as U[o][i]
 *   chi       maximum bond dimension kept (1 <= chi <= chi_max)
 *   svd_cutoff  singular values <= svd_cutoff * sigma_1 are dropped (e.g. 1e-14)
 *   eps_out   host float64 [n_gates] or NULL: gate error eps_i (Eq. 1) as the
 *             discarded fraction sum_{j>chi} s_j^2 / sum_j s_j^2; 0 for 1q gates
 * After the call the BP messages on the gated bonds equal diag(S)/|S| and the
 * others are stale until tns_bp_gauge runs.
 */
tns_status tns_apply_gate_layer(tns_state* s, int32_t n_gates, const int32_t* sites, const double* mats, int32_t chi,
                                double svd_cutoff, double* eps_out);

/*
 * tns_bp_gauge -- run belief propagation on <psi|psi> (Methods; Appendix Fig. 8c):
 * every message m_{v->v'} is replaced, in parallel, by psi_v psi_v^* contracted
 * with all messages into v except the one from v', Hermitised and normalised to
 * unit Frobenius norm, until max |m_new - m_old|_F < tol or max_iter sweeps.
 *   iters_out, residual_out  host pointers or NULL.
 * Precision: in TNS_PREC_FP64 every contraction is FP64.  In TNS_PREC_MIXED the
 * message contractions run on complex64 copies of the site tensors and messages
 * (TF32x3 tensor cores, FP32 accumulation) while the Hermitisation, normalisation,
 * residual and the stored messages stay FP64.  The residual of the mixed path cannot
 * fall much below the FP32 rounding of those contractions: a tol below 1e-6 is
 * raised to 1e-6, and a residual under 1e-3 that stops falling (less than a 10% gain
 * over its best for 5 iterations) counts as converged at that floor.
 * The host checks the residual of iteration i while iteration i + 1 runs, so
 * iters_out may exceed the first iteration below tol by one.
 * Returns TNS_ERR_NOT_CONVERGED (state still valid) when max_iter is reached.
 */
tns_status tns_bp_gauge(tns_state* s, int32_t max_iter, double tol, int32_t* iters_out, double* residual_out);

/*
 * tns_bp_stats -- measurements of the last tns_bp_gauge call on this state:
 *   device_ms  elapsed device time of all its iterations (CUDA events on the state's
 *              stream, from the first launch to the last residual copy)
 *   bytes      algorithmic bytes: per iteration and directed edge, the site tensor
 *              (read once for ket and bra), the incoming messages and the new message,
 *              in the path's element size (16 B FP64, 8 B mixed)
 *   flops      algorithmic real flops of the message contractions (8 per complex MAC)
 * Any pointer may be NULL.  All zero before the first call.
 */
tns_status tns_bp_stats(const tns_state* s, double* device_ms, double* bytes, double* flops);

/*
 * tns_sample -- draw n_samples bitstrings with the boundary-MPS sampler (Appendix,
 * Fig. 7d) at boundary rank chi_b (R_x = R_n = chi_b).  Rows of the (oriented)
 * grid are the partitions.  The norm environments are contracted once from the
 * bottom; each sample then absorbs row b into its boundary MPS, compresses it to
 * chi_b (zip-up sweep; truncated SVD of every site matrix by a range finder with
 * subspace iterations, see tns_set_compression), draws the row's qubits from
 * their one-site conditionals, and projects.
 *   seed      Philox4x32-10 key: qubit q of sample i uses counter
 *             (i lo, i hi, q, 0); x_q = 1 iff u >= q(0 | prefix)
 *   bits_dev  device uint8 [n_samples][n_sites] (caller-owned)
 *   logq_dev  device float64 [n_samples]: log q(x), sum of log conditionals
 *   cond_dev  device float64 [n_samples][n_sites] or NULL: q(x_q = 0 | prefix)
 * Deterministic for a given (state, chi_b, seed, precision).
 */
tns_status tns_sample(tns_state* s, int32_t chi_b, int64_t n_samples, uint64_t seed, uint8_t* bits_dev,
                      double* logq_dev, double* cond_dev);

/*
 * tns_sample_range -- samples first .. first + n_samples - 1 of the stream that
 * tns_sample draws for this (state, chi_b, seed): output row r holds sample
 * first + r (Philox counter (first + r, q)), equal to row first + r of a
 * tns_sample call with at least first + n_samples samples: bit-identical in
 * TNS_PREC_FP64; in TNS_PREC_MIXED the same bits with conditionals and log q equal
 * to FP32 rounding (a contraction whose rows span the chunk's samples may run on the
 * tensor cores or the CUDA cores depending on the chunk's size), so bits can differ
 * only where u and q(0 | prefix) tie to that rounding.  Samples are independent
 * draws, so disjoint ranges shard one stream across devices or calls with no
 * exchange between them.  first < 0 is TNS_ERR_ARG; buffers as tns_sample.
 */
tns_status tns_sample_range(tns_state* s, int32_t chi_b, int64_t first, int64_t n_samples, uint64_t seed,
                            uint8_t* bits_dev, double* logq_dev, double* cond_dev);

/*
 * tns_sample_replay -- like tns_sample, but the bits are given (bits_dev is read,
 * not written) and only the conditionals and log q along them are computed
 * (forced-path replay; used to verify samples and to score bitstrings under q).
 */
tns_status tns_sample_replay(tns_state* s, int32_t chi_b, int64_t n, uint64_t seed, const uint8_t* bits_dev,
                             double* logq_dev, double* cond_dev);

/*
 * tns_amplitude -- <x|psi> for n bitstrings by single-layer boundary MPS over the
 * projected rows at rank chi_b (Methods, "p(x) = |<x|psi>|^2"; Appendix).
 *   bits_dev     device uint8 [n][n_sites]
 *   log_abs_dev  device float64 [n]: log |<x|psi>| (-inf for an exact zero)
 *   phase_dev    device float64 [n]: arg <x|psi>
 */
tns_status tns_amplitude(tns_state* s, int32_t chi_b, int64_t n, const uint8_t* bits_dev, double* log_abs_dev,
                         double* phase_dev);

/*
 * tns_certify -- check sampled bitstrings against an independent contraction
 * (Methods, p(x) = |<x|psi>|^2 / <psi|psi>; Appendix, verification of the samples):
 * log p(x) from tns_amplitude and tns_log_norm at rank chi_b (e.g. twice the
 * sampling rank), and the statistics of w = p(x) / q(x) over the samples, which
 * average to 1 when q is the sampling distribution (importance-sampling identity).
 *   bits_dev    device uint8 [n][n_sites];  logq_dev  device float64 [n] (log q(x))
 *   logp_dev    device float64 [n]: log p(x) (-inf for an exact zero)
 *   stats_host  host float64 [5]: mean w, its standard error, mean(log q - log p)
 *               (the KL-divergence estimate of q from p), samples with p > 0, and
 *               log <psi|psi> at chi_b
 */
tns_status tns_certify(tns_state* s, int32_t chi_b, int64_t n, const uint8_t* bits_dev, const double* logq_dev,
                       double* logp_dev, double* stats_host);

/* Sum over applied two-qubit gates of log(1 - eps_i): log of the fidelity
 * estimate f of Eq. 2. */
tns_status tns_log_fidelity(const tns_state* s, double* log_f);

/* log <psi|psi> from the bottom norm environments at rank chi_b. */
tns_status tns_log_norm(tns_state* s, int32_t chi_b, double* log_norm);

/*
 * tns_direct_marginals -- sample-free marginals from the boundary-MPS contraction
 * of <psi|psi> (Methods, expectation values; Results Fig. 4): for every qubit
 * <n_q> = <psi|P1_q|psi> / <psi|psi>, P1 = |1><1|, and for every pair of qubits in
 * the same grid row <n_q n_q'>.  Each row is contracted exactly between its top
 * and bottom norm environments at rank chi_b (built as for tns_log_norm, the top
 * ones on the state read upside down).
 *   one_host  host float64 [n_sites]
 *   two_host  host float64 [n_sites][n_sites] or NULL: same-row pairs (and the
 *             diagonal, = one_host); NaN for pairs in different rows
 * Precision as set by tns_set_precision; the cost per row is about
 * 3 W + W^2 / 2 site steps of O(chi_b^3 chi^6) each.
 */
tns_status tns_direct_marginals(tns_state* s, int32_t chi_b, double* one_host, double* two_host);

/*
 * tns_set_graphs -- 1 (default): tns_sample and tns_sample_replay run each chunk's
 * launch sequence (several thousand kernels at the 10x10 workload) from a CUDA
 * graph.  The first chunk of a given shape runs eagerly, the second is captured,
 * later ones replay the graph; the seed, first sample index and output buffers are
 * read on the device, so one graph serves every call.  A graph is rebuilt when the
 * state, its precision, rank, compression settings, chunk size or any internal
 * buffer changes.  Results are identical with and without graphs.  0: always
 * launch eagerly (also the case while kernel timing is on).
 */
tns_status tns_set_graphs(tns_state* s, int32_t enable);

/* Select the precision of later tns_sample / tns_amplitude calls. */
tns_status tns_set_precision(tns_state* s, tns_prec prec);

/* Select how the mixed-precision path runs its contractions: 1 (default) =
 * every contraction of at least 2^24 complex multiply-adds on the tcgen05 tensor
 * cores, kind::tf32 with a three-pass hi/lo split product (FP32-level accuracy),
 * smaller ones on FP32 CUDA cores; 0 = all on FP32 CUDA cores.  Shapes the
 * tensor-core kernel does not support fall back to CUDA cores automatically. */
tns_status tns_set_tensor_cores(tns_state* s, int32_t enable);

/*
 * tns_set_compression -- settings of the truncated SVD in every zip-up compression
 * of tns_sample, tns_sample_replay, tns_amplitude and tns_log_norm (the "QR and
 * truncated SVD" of the boundary-MPS contraction; Methods and Appendix "Sampling
 * from a Tensor Network State").  The rank-chi_b truncation of each site matrix T
 * (M x N) is taken from a k = chi_b + oversample column range finder with
 * power_iters subspace iterations (env_power_iters for the norm environments):
 * the kept subspace differs from the exact truncated SVD's by a factor
 * ~(sigma_{k+1} / sigma_chi_b)^(2 q + 1), and k >= N gives the exact truncated SVD.
 * Defaults: oversample 48, power_iters 3, env_power_iters 6 (at the 10x10 chi = 16,
 * chi_b = 64 workload every conditional is then within 1.2e-4 of the exact
 * truncated SVD's; 8 and 1 give 1e-2).
 *   0 <= oversample <= 4096, 0 <= power_iters, env_power_iters <= 64.
 * Changing them rebuilds the cached norm environments on their next use.
 */
tns_status tns_set_compression(tns_state* s, int32_t oversample, int32_t power_iters, int32_t env_power_iters);

/* Query: grid rows/cols after orientation, whether it was transposed, and the
 * current maximum bond dimension. */
tns_status tns_query(const tns_state* s, int32_t* H, int32_t* W, int32_t* transposed, int32_t* chi_now);

/* Save / load the state (site tensors, bond dimensions, messages, log f) to a
 * little-endian binary file ("TNSF" format: header, then per grid cell its
 * physical and bond dimensions and complex128 entries in [s][u][l][d][r] order,
 * then the messages).  tns_load creates a new state on the given stream. */
tns_status tns_save(const tns_state* s, const char* path);
tns_status tns_load(const char* path, void* cuda_stream, tns_state** out);

/* Number of library kernel launches issued since the state was created. */
tns_status tns_launch_count(const tns_state* s, int64_t* launches);

/*
 * Kernel timing: when enabled, the sampler brackets each launch of its kernel
 * classes with CUDA events on the state's stream and accumulates, per class,
 * the elapsed device time, the launch count and the algorithmic FLOPs (8 per
 * complex multiply-add of the contraction as written, excluding any padding).
 * Classes: 0 = environment contractions (the row's norm-environment GEMMs of
 * the marginal sweeps), 1 = other marginal-sweep contractions, 2 = zip-up
 * compression contractions, 3 = FP64 factorisations (Cholesky, Jacobi), 4 =
 * fused marginal/draw/project kernel, 5/6/7 = tensor-core operand packing
 * (gathers and the real block expansion with TF32 remainders) for classes
 * 0/1/2, 8/9 = zip / other sweep contractions of the mixed path that ran on
 * the CUDA cores (too small for the tensor-core kernel).  With tensor cores
 * on, classes 0-2 time the GEMM kernel alone.  tns_profile_enable(s, 1) also
 * clears the counters.
 */
tns_status tns_profile_enable(tns_state* s, int32_t enable);
tns_status tns_profile_read(tns_state* s, int32_t kernel_class, double* device_ms, int64_t* launches,
                            double* flops);

/*
 * tns_eigh_noalloc -- batched Hermitian eigendecomposition (the library's FP64
 * parallel-Jacobi eigensolver, the same computation as tns_test_eigh in
 * tns_testing.h) that allocates no device memory.  The paper has no
 * counterpart; it serves callers that cannot call cudaMalloc, such as programs
 * whose device memory is owned by another allocator that has reserved HBM up
 * front, or latency-critical code that cannot accept the device-wide
 * synchronisation an allocation may imply.
 *   batch, n   number and order of the matrices (1 <= n <= 512)
 *   A_dev      device complex128 [batch][n][n], Hermitian, read only
 *   lam_dev    device float64 [batch][n]: eigenvalues, descending
 *   V_dev      device complex128 [batch][n][n]: column j is eigenvector j
 *   cuda_stream  stream to launch on; the call returns after the launch and the
 *              results are ready when the stream reaches that point
 * Scratch: a static 16 MiB device array per GPU that loads the library, held
 * until the process exits.  It holds 4 bytes per matrix plus, when the
 * eigensolver's shared-memory working copy, 2*n'*(n'+1)*16 bytes (n' = n rounded
 * up to even), exceeds 200 KiB, a global working copy of 2*n'^2*16 bytes per
 * matrix; a batch needing more than 16 MiB returns TNS_ERR_ARG.  Every call
 * shares the one array, so calls that overlap on the GPU (different streams,
 * or threads using one device) race: order them on one stream.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Convergence is not reported by this call (no host synchronisation): the
 * per-matrix status words stay in the scratch for tns_eigh_noalloc_status.
 */
tns_status tns_eigh_noalloc(int32_t batch, int32_t n, const double* A_dev, double* lam_dev, double* V_dev,
                            void* cuda_stream);

/*
 * tns_eigh_noalloc_status -- the convergence status of the last tns_eigh_noalloc
 * call on the current device, as a stream-ordered device-to-device copy (no
 * allocation, no host wait): status_dev (device int32 [batch], caller-owned)
 * receives, per matrix, 0 if the Jacobi sweeps converged and 1 if they stopped at
 * the sweep cap (the condition the allocating entry points return as
 * TNS_ERR_NUMERIC).  Issue it on the stream of that call and before the next one;
 * batch above the last call's batch returns TNS_ERR_ARG.  The paper has no
 * counterpart.
 */
tns_status tns_eigh_noalloc_status(int32_t batch, int32_t* status_dev, void* cuda_stream);

/*
 * Learned proposal and independent Metropolis-Hastings.  The paper samples only
 * with the boundary-MPS sampler above; these calls add an optional second stage:
 * a MADE network (masked autoregressive MLP: Germain, Gregor, Murray and
 * Larochelle, ICML 2015) fitted by maximum likelihood to the sampler's
 * bitstrings, whose cheap exact samples and log-probabilities log g(x) feed an
 * independent Metropolis-Hastings chain with target p(x) = |<x|psi>|^2 (log p
 * from tns_amplitude).
 *
 * Network: n inputs in natural qubit order, three ReLU hidden layers of width h,
 * n logits; g(x_i = 1 | x_<i) = sigmoid(l_i).  Degrees: input/output i -> i+1,
 * hidden unit k -> 1 + (k mod (n-1)).  Hidden masks keep weight (k, j) iff
 * deg(k) >= deg(j); the output mask keeps (i, k) iff i+1 > deg(k).  Parameters
 * are packed float32: W1[h][n], b1[h], W2[h][h], b2[h], W3[h][h], b3[h],
 * W4[n][h], b4[n] (P = 2hn + 2h^2 + 3h + n floats).
 * Arithmetic: FP32 master weights and Adam moments; GEMM operands (masked
 * weights, activations, back-propagated errors) rounded to BF16, products
 * accumulated in FP32; log g and the MH acceptance test in FP64.
 * Bit buffers are device uint8 [rows][n], one byte per qubit (0 or 1).
 * A tns_made is used by one host thread at a time and runs on the stream given
 * at creation; every call returns after that stream has finished the call's work.
 */
typedef struct tns_made tns_made; /* opaque, library-owned */

/*
 * tns_made_create -- allocate a network with the given initial parameters.
 *   n_sites >= 2, hidden >= 1; params_host  host float32 [P], copied.
 *   cuda_stream  stream for every later call on this network.
 */
tns_status tns_made_create(int32_t n_sites, int32_t hidden, const float* params_host, void* cuda_stream,
                           tns_made** out);

/* tns_made_params -- copy the current FP32 parameters to params_host [P]. */
tns_status tns_made_params(const tns_made* m, float* params_host);

/*
 * tns_made_train -- mini-batch Adam (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the
 * mean negative log-likelihood.  Epoch e visits the rows of bits_dev [n][n_sites]
 * in the order orders_host[e*n .. e*n+n-1] (host int32, NULL = natural order),
 * in consecutive batches of `batch` rows (the last may be shorter).  The Adam
 * step count carries over between calls.  loss_host (host float64 [epochs] or
 * NULL) receives, per epoch, the mean NLL of each row under the parameters
 * before the step of its batch.
 */
tns_status tns_made_train(tns_made* m, const uint8_t* bits_dev, int64_t n, int32_t batch, int32_t epochs,
                          const int32_t* orders_host, float lr, double* loss_host);

/*
 * tns_made_grad -- gradient of the mean NLL over the n rows of bits_dev
 * (1 <= n <= 2^20) into grad_host (host float32 [P], or NULL); the mean NLL into
 * *loss (or NULL).  Masked-out weights get gradient 0.  Parameters unchanged.
 */
tns_status tns_made_grad(tns_made* m, const uint8_t* bits_dev, int64_t n, float* grad_host, double* loss);

/* tns_made_logprob -- log g(x) (device float64 [n]) of the n rows of bits_dev. */
tns_status tns_made_logprob(tns_made* m, const uint8_t* bits_dev, int64_t n, double* logg_dev);

/*
 * tns_made_sample -- n ancestral samples into bits_dev [n][n_sites] and their
 * log g into logg_dev [n].  Qubit i of sample s is 1 iff u >= g(x_i = 0 | x_<i),
 * u = the 53-bit uniform of Philox4x32-10 words (0, 1) at counter
 * (s mod 2^32, s div 2^32, i, 1) under key (seed mod 2^32, seed div 2^32).
 */
tns_status tns_made_sample(tns_made* m, int64_t n, uint64_t seed, uint8_t* bits_dev, double* logg_dev);

void tns_made_destroy(tns_made* m);

/*
 * tns_mh_independent -- n_chains independent Metropolis-Hastings chains over
 * precomputed proposals.  Chain c at step t proposes proposal (c, t) with target
 * log-probability logp_prop_dev[c*n_steps+t] and proposal log-probability
 * logg_prop_dev[...] (device float64 [n_chains][n_steps]); the chain starts
 * from a state with log p = logp0_dev[c], log g = logg0_dev[c].  The proposal is
 * accepted iff log u < (lp' - lp) + (lg - lg'), u as in tns_made_sample at
 * counter (c, t, 0, 2) (u = 0 always accepts).  Outputs: state_dev (device int32
 * [n_chains][n_steps]) = index t' of the proposal chain c holds after step t,
 * -1 while it holds its initial state; accepted_dev (device int64 [n_chains]) =
 * accepted moves.  Log-probabilities may be unnormalised (constants cancel).
 */
tns_status tns_mh_independent(int32_t n_chains, int32_t n_steps, const double* logp_prop_dev,
                              const double* logg_prop_dev, const double* logp0_dev, const double* logg0_dev,
                              uint64_t seed, int32_t* state_dev, int64_t* accepted_dev, void* cuda_stream);

void tns_destroy(tns_state* s);
const char* tns_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TNS_H */
