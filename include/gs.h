/*
 * gs.h - C ABI of the GaloisSAT differentiable solving stage on B300 (sm_103a).
 *
 * Method (arXiv 2603.28796, Sec. "Differentiable SAT Formulation"): a CNF formula's clauses
 * become polynomials C_t = 1 - prod_i (1 - s_i) over literal values s_i (Eq. 1, Eq. 2); each
 * variable is relaxed to x = sigma(delta / tau), delta being the difference of the two logits of
 * the two Boolean states (Eq. 3 without noise); the loss is the MaxSAT sum of Eq. 5, kept here
 * in its non-negative form L_unsat = sum_t prod_i (1 - s_i) = m + L (same gradient, zero exactly
 * at satisfying Boolean points); Adam updates delta (Sec. "Experiment Setup": Adam, lr 0.5 on
 * the two logits == lr 1.0 on delta); rounding is the argmax of Eq. 4, x_hat = [delta > 0].
 *
 * Conventions shared by every call below.
 *  - Variables and candidates. A problem has n variables (summed over its instances). A batch
 *    of B candidate assignments is stored var-major: element (v, b) of an array with row
 *    stride ldB is at index v * ldB + b. ldB >= B, and every row must start on a 16-byte
 *    boundary: ldB a multiple of 4 for float arrays, of 8 for 16-bit relaxed values (the
 *    float arrays used with them share that ldB). Columns [B, ldB) are never written.
 *  - Memory. Pointers marked "device" are CUDA device pointers owned by the caller, 16-byte
 *    aligned (8-byte for double arrays, 4-byte for int32 ones); "host" pointers are read during
 *    the call only. The library owns only the problem's index structures and a workspace that
 *    grows on demand (see gs_reserve).
 *  - Streams. gs_stream is a cudaStream_t (NULL = legacy default stream). Every compute call
 *    only enqueues work on the stream and returns; results are ready when the stream is.
 *  - Errors. Invalid arguments are rejected before anything is enqueued and leave outputs
 *    untouched. Errors raised on the device (a bounded wait that timed out) are sticky and are
 *    reported by gs_sync_status. Nothing crosses the ABI as an exception.
 *  - Determinism. No floating-point atomics are used: for a given problem, B, dtype and GPU,
 *    every output is bitwise reproducible.
 *  - Limits. Clause width <= 256 literals; n < 2^28 - 2 variables; B <= 2^30.
 */
#ifndef GALOISSAT_GS_H
#define GALOISSAT_GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad pointer, size, stride, alignment, literal or instance map */
    GS_ERR_PARSE = 2,       /* malformed DIMACS text */
    GS_ERR_OOM = 3,         /* host or device allocation failed */
    GS_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed (see gs_last_error) */
    GS_ERR_UNSUPPORTED = 5, /* beyond the limits above */
    GS_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up (from gs_sync_status) */
    GS_ERR_STATE = 7        /* wrong device, or workspace growth requested during stream capture */
} gs_status;

/* Storage type of the relaxed values x (the arrays the clause products gather from). The
 * logits delta and the Adam moments are always float32; products accumulate in float32. */
typedef enum { GS_F32 = 0, GS_BF16 = 1, GS_F16 = 2 } gs_dtype;

typedef void* gs_stream; /* cudaStream_t */
typedef struct gs_problem gs_problem;

/* Problem statistics (gs_info_get, gs_inspect_cnf). */
typedef struct {
    int64_t n_vars;       /* variables, all instances */
    int64_t n_clauses;    /* clauses, all instances */
    int64_t nnz;          /* literal occurrences */
    int32_t n_inst;       /* instances (1 for gs_load_cnf) */
    int32_t max_k;        /* widest clause */
    int64_t n_empty;      /* empty clauses (always unsatisfied, U_t = 1) */
    int64_t n_unit;       /* clauses with one literal */
    int64_t n_taut;       /* clauses containing some x and NOT x (kept and evaluated as written) */
    int64_t n_dup;        /* clauses repeating a literal (each copy is its own factor) */
    int64_t n_occ_codes;  /* size of the variable-major occurrence lists */
    int64_t n_fwd_tiles;  /* clause tiles (forward, check) */
    int64_t n_var_tiles;  /* occurrence tiles (backward, fused step) */
    int64_t n_split;      /* variables whose occurrences are split over several tiles */
    int64_t device_bytes; /* index structures held on the device */
    int32_t fwd_tile_codes;  /* tile caps the problem was built with (gs_plan_opts) */
    int32_t var_tile_codes;
    int32_t own_item_codes;
    int32_t reserved;
} gs_info;

/* Adam hyper-parameters on delta. Defaults (gs_adam_default): lr 1.0, beta1 0.9, beta2 0.999,
 * eps 1e-8, tau 1.0 - PyTorch's Adam defaults with the paper's lr 0.5 carried over from the
 * two logits (theta_1, theta_0) to their difference delta, and the paper's tau = 1. Given in
 * double precision: 1 - beta and the bias corrections are formed in double on the host and
 * rounded once to float32 for the kernels (as PyTorch does with its Python-float scalars). */
typedef struct {
    double lr, beta1, beta2, eps, tau;
} gs_adam;

/* Fills *out with the defaults above. */
void gs_adam_default(gs_adam* out);

/*
 * gs_load_cnf - build a problem from one CNF in CSR form (Sec. "Differentiable SAT
 * Formulation": the clause set the polynomials of Eq. 2 are taken over).
 *   n_vars      variables, literals refer to 1..n_vars.
 *   n_clauses   clauses m.
 *   clause_ptr  host [m + 1], clause_ptr[0] = 0, non-decreasing; clause t holds
 *               lits[clause_ptr[t] .. clause_ptr[t+1]).
 *   lits        host [clause_ptr[m]], DIMACS literals: +v for x_v, -v for NOT x_v, 1 <= v <= n.
 *   stream      stream used for the uploads (the call returns after they complete).
 *   out         receives the problem handle (owned by the caller, freed with gs_free).
 * Builds on the device the clause->literal CSR (clause tiles), its transpose var->occurrence
 * lists (occurrence tiles; each occurrence lists the other literals of its clause), and the
 * tile schedules. Empty, unit, tautological and duplicate-literal clauses are kept and
 * evaluated literally. Errors: GS_ERR_INVALID_ARG (null pointer, negative size, non-monotone
 * clause_ptr, literal 0 or out of range), GS_ERR_UNSUPPORTED (limits), GS_ERR_OOM, GS_ERR_CUDA.
 */
gs_status gs_load_cnf(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                      gs_stream stream, gs_problem** out);

/*
 * gs_load_batch - many independent instances in one problem (the paper's batched training of
 * many candidates, extended to many formulas of uneven size in one launch).
 *   n_inst         instances.
 *   n_vars         host [n_inst], variables of each instance (literals are instance-local,
 *                  1..n_vars[i]).
 *   n_clauses      host [n_inst], clauses of each instance.
 *   clause_ptr     host [sum n_clauses + 1], one CSR over the concatenated clauses.
 *   lits           host [clause_ptr[end]], instance-local DIMACS literals.
 * Instance i owns candidate rows [sum_{j<i} n_vars[j], + n_vars[i]) of every candidate array
 * and row i of every per-instance output ([n_inst][B] losses and unsat counts, best[n_inst]).
 * Tiles never cross instances. Errors as gs_load_cnf.
 */
gs_status gs_load_batch(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                        const int32_t* lits, gs_stream stream, gs_problem** out);

/*
 * gs_plan_opts - tile sizes of the index structures (a tuning knob of the kernels' work items,
 * fixed when a problem is built; 0 takes the default).
 *   fwd_tile_codes  literal codes per clause tile (forward pass, check): 32..512, default 512.
 *   var_tile_codes  occurrence codes per occurrence tile (backward, fused step): 32..384,
 *                   default 384; a variable with more codes is split over several tiles.
 *   own_item_codes  target codes per owned-variable work item: 256..65536, default 4096.
 *   reserved        must be 0.
 * A tile always holds at least one whole clause / occurrence. Results differ between tilings only
 * in the float32 summation order of the loss.
 */
typedef struct {
    int32_t fwd_tile_codes;
    int32_t var_tile_codes;
    int32_t own_item_codes;
    int32_t reserved;
} gs_plan_opts;

/*
 * gs_load_batch_opts - gs_load_batch with explicit tile sizes (opts may be NULL: defaults).
 * Errors: as gs_load_batch, plus GS_ERR_INVALID_ARG for caps out of range.
 */
gs_status gs_load_batch_opts(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses,
                             const int64_t* clause_ptr, const int32_t* lits, const gs_plan_opts* opts,
                             gs_stream stream, gs_problem** out);

/*
 * gs_load_dimacs - gs_load_cnf from a DIMACS CNF text file (header "p cnf n m", clauses
 * terminated by 0, comment lines starting with 'c'). Errors: GS_ERR_PARSE on malformed text or
 * a clause count that disagrees with the header, then as gs_load_cnf.
 */
gs_status gs_load_dimacs(const char* path, gs_stream stream, gs_problem** out);

/*
 * gs_inspect_cnf - validate a CSR formula and compute its gs_info fields (no device work; the
 * tile counts and device_bytes are those gs_load_cnf would build). Errors as gs_load_cnf.
 */
gs_status gs_inspect_cnf(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                         gs_info* out);

/*
 * gs_tseitin3 - the paper's width normalisation (Sec. "Clause Normalization for Vectorization",
 * Eq. 6-8, host only, no device work): every clause of u > 3 literals becomes the chain
 *   (l1 v l2 v f1) (-f1 v l3 v f2) ... (-f_{u-3} v l_{u-1} v l_u)
 * over fresh variables f numbered n_vars + 1, n_vars + 2, ... in clause order; a clause of 1 or
 * 2 literals repeats its last literal to width 3 (the appendix's (-x1 v x3 v x3)); width 3 is
 * kept and an empty clause stays empty. The result is equisatisfiable with the input and its
 * first n_vars variables are the input's. Call once with clause_ptr_out = lits_out = NULL to get
 * *n_out, *m_out, *nnz_out, then with host buffers of m_out + 1 and nnz_out entries.
 * Errors: as gs_inspect_cnf.
 */
gs_status gs_tseitin3(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                      int64_t* n_out, int64_t* m_out, int64_t* nnz_out, int64_t* clause_ptr_out, int32_t* lits_out);

/* gs_info_get - statistics of a loaded problem. GS_ERR_INVALID_ARG on null arguments. */
gs_status gs_info_get(const gs_problem* prob, gs_info* out);

/*
 * gs_reserve - size the workspace for batches of B candidates stored as dtype, so that later
 * calls with (B, dtype) allocate nothing (required before capturing them in a CUDA graph).
 * Synchronous. Errors: GS_ERR_INVALID_ARG, GS_ERR_OOM.
 */
gs_status gs_reserve(gs_problem* prob, int32_t B, gs_dtype dtype);

/*
 * Tuning of the tiled kernels. Each lane handles 4 (float32) or 8 (16-bit) consecutive
 * candidates and a candidate chunk spans up to `lanes` lanes; the kernels sweep all tiles once
 * per chunk, so the rows of relaxed values gathered during a sweep are n x chunk wide. A
 * smaller cap keeps that working set inside L2 at the price of more sweeps over the tiles.
 *   var_lanes  cap for the variable-major pass (gs_backward, gs_step): 0 (= 32), 4, 8, 16, 32.
 *   fwd_lanes  cap for the clause-major forward (gs_forward): 0 (= 32), 4, 8, 16, 32.
 *   var_gather how the variable-major pass fetches the rows its occurrence codes name:
 *              0 = automatic (currently per-lane register loads), 1 = per-lane register loads,
 *              2 = TMA tile::gather4 copies into a shared-memory ring when a chunk spans 32
 *              lanes (register loads otherwise).
 *   loss_mode  how the fused step (gs_step with grad = NULL) produces its loss: 0 = automatic
 *              (currently 1), 1 = credited inside the variable-major pass at each clause's first
 *              literal, 2 = a separate clause-major forward pass on x_in (fewer instructions in the
 *              variable pass; faster for wide clauses and small candidate rows).
 *   var_split  how the lane groups of a warp share the variable-major pass when a candidate
 *              chunk spans fewer than 32 lanes (small B): 0 = automatic (currently 1), 1 = all
 *              groups work on one variable at a time, splitting its occurrences (tiles staged in
 *              shared memory by TMA), 2 = each group owns whole variables of a run of variables
 *              cut at equal code counts (codes read from global memory; no per-variable
 *              reduction across groups, less padding of the gather batches).
 * Results do not depend on the tuning beyond float32 summation order. Call gs_reserve again
 * after changing it if later calls are captured in a CUDA graph.
 */
typedef struct {
    int32_t var_lanes;
    int32_t fwd_lanes;
    int32_t var_gather;
    int32_t loss_mode;
    int32_t var_split;
} gs_tuning;

/* gs_set_tuning / gs_get_tuning - set or read the caps above. Errors: GS_ERR_INVALID_ARG. */
gs_status gs_set_tuning(gs_problem* prob, const gs_tuning* tuning);
gs_status gs_get_tuning(const gs_problem* prob, gs_tuning* tuning);

/*
 * gs_autotune - pick the tuning for batches of B candidates stored as dtype by timing the fused
 * step (gs_step with grad = NULL and a loss) over the candidates-per-warp choices (lanes per
 * chunk) and both gather modes, gs_forward over its lanes per chunk, and the two loss modes of
 * the fused step, on temporary buffers
 * it allocates and frees (n x B of each array). The fastest setting is applied to the problem
 * (gs_set_tuning), written to *out when out is not NULL, and the workspace is reserved for it.
 * Synchronous; not allowed during stream capture (GS_ERR_STATE). Errors: GS_ERR_INVALID_ARG,
 * GS_ERR_OOM, GS_ERR_CUDA.
 */
gs_status gs_autotune(gs_problem* prob, int32_t B, gs_dtype dtype, gs_stream stream, gs_tuning* out);

/*
 * gs_relax - relaxed values x = sigma(delta / tau) (Eq. 3 with two states and no Gumbel
 * noise), rounded to nearest-even when dtype is 16-bit.
 *   delta  device float [n][ldB] (input).   x  device dtype [n][ldB] (output).
 * Errors: GS_ERR_INVALID_ARG (null, alignment, ldB, tau <= 0).
 */
gs_status gs_relax(gs_problem* prob, const float* delta, void* x, gs_dtype dtype, int32_t B, int64_t ldB, float tau,
                   gs_stream stream);

/*
 * gs_forward - per-candidate loss of Eq. 2 + Eq. 5 at relaxed values x:
 *   loss[i][b] = sum over clauses t of instance i of prod_{literals of t} f, f = 1 - x_v for a
 *   positive literal and x_v for a negated one (= m_i + L_paper, L_paper = -sum_t C_t).
 *   x     device dtype [n][ldB] (input).   loss  device double [n_inst][B] (output).
 * Clause products accumulate in float32 (compensated within a tile); tiles are summed in
 * float64 in a fixed order. Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_forward(gs_problem* prob, const void* x, gs_dtype dtype, int32_t B, int64_t ldB, double* loss,
                     gs_stream stream);

/*
 * gs_forward_noalloc - gs_forward for callers that must not allocate device memory. Some host
 * programs cannot call cudaMalloc while they run: a process whose device memory is entirely
 * pre-reserved by another allocator (a serving stack or framework caching allocator), code that
 * runs while another component is capturing or replaying work on the device, or a latency-bound
 * loop that cannot afford the device-wide synchronisation an allocation may cause. gs_forward
 * may grow the problem's workspace on first use; this variant never allocates or frees memory.
 * The paper has no counterpart: this is an operational variant of gs_forward.
 *   Arguments and output are those of gs_forward. It runs gs_forward's kernels with the same
 *   chunking (the problem's tuned lanes per chunk) and the same two-stage reduction order, so
 *   its results are bitwise those of gs_forward on the same problem, tuning and input.
 *   Scratch: a fixed device array inside the library, present on every GPU that loads the
 *   library until the process exits: 16 MiB of per-tile partial sums, n_fwd_tiles (gs_info) x
 *   Bpad x 4 bytes (Bpad: B rounded up to the candidate chunk, at most 128 float32 / 256 16-bit
 *   candidates per chunk), 4 MiB of stage-1 sums (reduction segments x instances x B x 8 bytes;
 *   at most 256 segments of at least 32 tiles each), and a 256-byte counter block. Larger
 *   requests are rejected with GS_ERR_UNSUPPORTED and a message naming the limit.
 *   The first call on a device looks up the array's device address (with that device current);
 *   make that first call before any stream capture. All calls on a device share the array and
 *   leave their partials in it: calls that overlap on the GPU (other streams, other problems,
 *   other host threads) race and must be serialised by the caller.
 * Errors: as gs_forward, plus GS_ERR_UNSUPPORTED when the request exceeds the scratch.
 */
gs_status gs_forward_noalloc(gs_problem* prob, const void* x, gs_dtype dtype, int32_t B, int64_t ldB, double* loss,
                             gs_stream stream);

/*
 * gs_backward - gradient of the loss above with respect to x (back-propagation through
 * Eq. 2; the paper's dashed backward arrows):
 *   grad[v][b] = w_b * sum over occurrences (t, i) of v of  sign_i * prod_{j in t, j != i} f_j,
 *   sign_i = -1 for a positive literal, +1 for a negated one; the leave-one-out product is the
 *   prefix product before i times the suffix product after i (exact at zeros, no division);
 *   w_b = dloss[inst(v)][b], or 1 when dloss is NULL.
 *   x      device dtype [n][ldB].   dloss  device double [n_inst][B] or NULL.
 *   grad   device float [n][ldB] (output; every (v, b < B) is written).
 * Each variable's gradient is gathered over its occurrence list (no atomics).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_backward(gs_problem* prob, const void* x, gs_dtype dtype, int32_t B, int64_t ldB, const double* dloss,
                      float* grad, gs_stream stream);

/*
 * gs_step - one Adam step on delta (Sec. "Experiment Setup"), in place:
 *   g = dL/dx * sigma(delta/tau) sigma(-delta/tau) / tau,  m = b1 m + (1-b1) g,
 *   v = b2 v + (1-b2) g^2,  delta -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps),
 *   x_out = sigma(delta / tau) (Eq. 3),  bits = [delta > 0] (Eq. 4).
 *   delta, m, v  device float [n][ldB], read and written.
 *   grad         device float [n][ldB] holding dL/dx, or NULL for the fused path: the
 *                gradient is formed from x_in in registers (gs_backward's arithmetic), never
 *                stored, and the update follows in the same kernel.
 *   x_in         device dtype [n][ldB]: the relaxed values the fused gradient is taken at
 *                (normally sigma(delta/tau) from the previous step); ignored when grad != NULL.
 *   x_out        device dtype [n][ldB] (output); must not overlap x_in. May be NULL only
 *                when grad != NULL.
 *   step         1-based Adam step t (bias correction).
 *   adam         hyper-parameters, NULL = defaults.
 *   loss         fused path only: device double [n_inst][B] receiving the loss at x_in (each
 *                clause's product is credited once, at its first literal), or NULL.
 *   bits         device uint64 [n][ceil(B/64)] receiving the rounded new delta (bit b%64 of word
 *                b/64 of row v is [delta > 0]; bits >= B are 0), or NULL.
 * Errors: GS_ERR_INVALID_ARG (also loss != NULL with grad != NULL), GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_step(gs_problem* prob, float* delta, float* m, float* v, const float* grad, const void* x_in, void* x_out,
                  gs_dtype dtype, int32_t B, int64_t ldB, int64_t step, const gs_adam* adam, double* loss,
                  uint64_t* bits, gs_stream stream);

/*
 * gs_round_check - round (Eq. 4: x_hat = [delta > 0], ties to 0) and check every clause exactly
 * in integer arithmetic (Eq. 2 at Boolean points: C_t = 1 iff some literal is true).
 *   delta  device float [n][ldB].
 *   bits   device uint64 [n][ceil(B/64)] receiving x_hat, or NULL (library workspace).
 *   unsat  device int32 [n_inst][B]: number of unsatisfied clauses of each candidate.
 *   best   device int32 [n_inst]: lowest candidate with the fewest unsatisfied clauses, or NULL.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_round_check(gs_problem* prob, const float* delta, int32_t B, int64_t ldB, uint64_t* bits, int32_t* unsat,
                         int32_t* best, gs_stream stream);

/*
 * gs_check_bits - the check half of gs_round_check on assignments already packed as above
 * (e.g. by gs_step's bits output). bits is read-only. Errors as gs_round_check.
 */
gs_status gs_check_bits(gs_problem* prob, const uint64_t* bits, int32_t B, int32_t* unsat, int32_t* best,
                        gs_stream stream);

/*
 * Straight-through Gumbel training (Sec. "Gradient-based Optimization with Gumbel-Softmax":
 * Eq. 3 with noise, Eq. 4 in the forward pass). With two logits per variable, Eq. 3 puts
 * y = sigma((delta + l) / tau) on state 1, delta = theta_1 - theta_0 and l = g_1 - g_0, which is
 * Logistic(0,1) for independent Gumbel(0,1) draws g. The forward pass uses the hard assignment
 * x_hat = [delta + l > 0] (ties to state 0); the backward pass takes dL/dx at x_hat (an integer:
 * negated occurrences of the variable whose other literals are all false, minus positive ones)
 * through the soft y: dL/d delta = dL/dx(x_hat) * y (1 - y) / tau. The loss at x_hat is the
 * number of unsatisfied clauses (gs_check_bits on x_hat).
 *
 * Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with key (seed mod 2^32, seed / 2^32)
 * and counter (b / 4, row, step mod 2^32, step / 2^32); candidate b takes output word b % 4;
 * k = word >> 9, u = (k + 1/2) 2^-23, l = log(u / (1 - u)) in float32. Rows are the batch's
 * variable rows (instances concatenated). The decision [delta + l > 0] in float32 is exact.
 */

/*
 * gs_st_noise - the logistic noise l of one step into noise, device float [n][ldB] (every
 * (v, b < B) written; 16-byte aligned; ldB a multiple of 4). step >= 0.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_st_noise(gs_problem* prob, uint64_t seed, int64_t step, float* noise, int32_t B, int64_t ldB,
                      gs_stream stream);

/*
 * gs_st_sample - hard assignment of a step: bits = [delta + l > 0] (Eq. 4 on the noisy logits).
 *   delta  device float [n][ldB].
 *   noise  device float [n][ldB] holding l, or NULL: l generated from (seed, step) as above.
 *   bits   device uint64 [n][ceil(B/64)] (output; bits >= B are 0).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_st_sample(gs_problem* prob, const float* delta, const float* noise, uint64_t seed, int64_t step,
                       int32_t B, int64_t ldB, uint64_t* bits, gs_stream stream);

/*
 * gs_st_step - one straight-through Gumbel training step t, in place:
 *   gx = dL/dx at bits_in (the hard assignment of step t, from gs_st_sample or the previous
 *   gs_st_step), y = sigma((delta + l_t)/tau), g = gx y (1 - y) / tau, Adam on delta exactly as
 *   gs_step, then bits_out = [delta' + l_{t+1} > 0], the hard assignment of step t + 1.
 *   delta, m, v          device float [n][ldB], read and written.
 *   bits_in              device uint64 [n][ceil(B/64)], read; bits_out the same shape, written
 *                        (every row; bits >= B are 0); they must not overlap.
 *   noise, noise_next    device float [n][ldB] holding l_t and l_{t+1}, or NULL: generated from
 *                        (seed, step) and (seed, step + 1) inside the kernel.
 *   noise_next_out       device float [n][ldB] receiving the generated l_{t+1} (noise_next must
 *                        be NULL), or NULL. Passing it back as the next step's noise draws each
 *                        value once instead of twice (a two-buffer ring).
 *   step                 1-based Adam step t (bias correction) and noise counter.
 * Gathers one bit per (literal, candidate): each variable's gradient is a signed bit-sliced
 * count over its occurrence list (no atomics).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_st_step(gs_problem* prob, float* delta, float* m, float* v, const uint64_t* bits_in, uint64_t* bits_out,
                     const float* noise, const float* noise_next, float* noise_next_out, uint64_t seed, int64_t step,
                     int32_t B, int64_t ldB, const gs_adam* adam, gs_stream stream);

/*
 * Candidate pool (Sec. "Partial Assignment Extraction for SAT Instances", the pool of Eq. 9) and
 * branching variables (Sec. "Guided Branching for UNSAT Instances"), from one trained candidate's
 * logits delta (the selected batch): row v of it is delta[v * stride] (a column of a [n][ldB]
 * array: pass delta + b_sel and stride ldB). Only rows 0 .. n_rows - 1 take part (the formula's
 * own variables when fresh chain variables follow them, Eq. 6-8).
 * Confidence of variable v in a sample is max_j y_j = sigma(|delta_v + l| / tau); it is ranked by
 * |delta_v + l| (the same order; float32 sigma would tie everything beyond |z| = 17), ties to the
 * lower row, so the result does not depend on tau.
 *
 * gs_pool_sample - N samples x^(k) = [delta + l^(k) > 0] with independent logistic noise and, for
 * each, the S rows of highest confidence.
 *   noise  device float [n_rows][ldN] (ldN >= N) holding l, or NULL: drawn from the generator of
 *          gs_st_noise with this seed and step 0, sample k in the place of candidate k.
 *   bits   device uint64 [n_rows][ceil(N/64)] receiving the samples (bits >= N zero), or NULL.
 *   sel    device int32 [N][S] receiving each sample's selected rows, ascending.
 *   1 <= S <= min(n_rows, 8192); 1 <= N <= 2^20. Uses a library workspace of 256 KiB per sample.
 * gs_branch_vars - the d rows of lowest confidence sigma(|delta_v| / tau), i.e. smallest |delta_v|
 *   (ties to the lower row), ascending in vars (device int32 [d]); 1 <= d <= min(n_rows, 8192).
 * Both are asynchronous on the stream. The unit clauses (x_v if the sample's bit is 1, else
 * not x_v) for each selected row, or the 2^d sign patterns of the branching rows, are added to
 * the formula by the host (a DIMACS writer is in the Python package).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED (S or d beyond 8192), GS_ERR_OOM, GS_ERR_STATE,
 * GS_ERR_CUDA.
 */
gs_status gs_pool_sample(gs_problem* prob, const float* delta, int64_t stride, int32_t n_rows, const float* noise,
                         int64_t ldN, uint64_t seed, int32_t N, int32_t S, uint64_t* bits, int32_t* sel,
                         gs_stream stream);
gs_status gs_branch_vars(gs_problem* prob, const float* delta, int64_t stride, int32_t n_rows, int32_t d,
                         int32_t* vars, gs_stream stream);

/*
 * gs_gather_probe - measurement kernel for the roofline of the variable-major pass (the K7 probe
 * of the measurement plan; no counterpart in the paper): n_gathers random row reads of row_bytes
 * bytes each, 16 bytes per lane, row_bytes / 16 lanes per row, 8 reads in flight per lane, with
 * the load form of the pass's gathers (16-byte non-coherent loads). Row k is at src + idx[k] * row_stride; an
 * index >= n_rows is skipped (no read). The loaded words are folded into *sink (XOR, one atomic
 * per warp) so that the reads are not removed. Time it with events to get the random-row gather
 * rate of the memory hierarchy at that row size and working set (n_rows x row_bytes).
 *   src   device, 16-byte aligned, n_rows rows of row_stride bytes (input, read only).
 *   idx   device uint32 [n_gathers] (input).   sink  device uint32 [1] (in/out).
 *   row_bytes a power of two in 16..512; row_stride a multiple of 16, >= row_bytes.
 * Errors: GS_ERR_INVALID_ARG (sizes, null, alignment), GS_ERR_CUDA.
 */
gs_status gs_gather_probe(const void* src, int64_t n_rows, int64_t row_stride, int32_t row_bytes, const uint32_t* idx,
                          int64_t n_gathers, uint32_t* sink, gs_stream stream);

/*
 * gs_wait_selftest - exercises the device-side failure path: one warp waits on a barrier phase
 * that nothing completes, gives up after limit_us microseconds (1..1e7) and records
 * GS_ERR_TIMEOUT in the problem's sticky status, exactly as a stalled tile copy would. No
 * memory is touched and the context stays usable; the next gs_sync_status returns
 * GS_ERR_TIMEOUT and clears it. Errors: GS_ERR_INVALID_ARG, GS_ERR_STATE, GS_ERR_CUDA.
 */
gs_status gs_wait_selftest(gs_problem* prob, uint32_t limit_us, gs_stream stream);

/*
 * gs_sync_status - waits for all work on the problem's device, then reports and clears the
 * sticky device-side status: GS_ERR_TIMEOUT if a bounded wait gave up since the last call
 * (the outputs of that call are incomplete), GS_ERR_CUDA on an asynchronous CUDA error, else
 * GS_OK.
 */
gs_status gs_sync_status(gs_problem* prob);

/* gs_free - releases the problem and its device memory (after synchronising). NULL is a no-op. */
void gs_free(gs_problem* prob);

/* gs_status_str - static description of a status code. */
const char* gs_status_str(gs_status status);

/* gs_last_error - thread-local text of the last error raised in this thread ("" if none). */
const char* gs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GALOISSAT_GS_H */
