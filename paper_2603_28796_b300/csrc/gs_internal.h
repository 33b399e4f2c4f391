// Internal layout shared by the host loader (gs_host.cu) and the kernels (gs_kernels.cu).
// Not part of the public C ABI (include/gs.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gs {

// ---------------------------------------------------------------------------------------------
// Limits of this implementation.
constexpr int kMaxClauseWidth = 256;            // literals per clause (8-bit fields in the tiles)
constexpr int64_t kMaxVars = (1LL << 28) - 2;   // 28-bit variable field in occurrence codes

// Forward / check tiles (clause-major). A tile holds whole clauses.
constexpr int kFwdCodes = 512;     // literal codes per tile
constexpr int kFwdClauses = 256;   // clauses per tile
// Occurrence tiles (variable-major). A tile holds whole variables, or one part of a variable
// whose occurrence list alone exceeds kVarCodes.
constexpr int kVarCodes = 384;     // occurrence codes per tile
constexpr int kVarVars = 64;       // variables per tile
constexpr int kOwnCodes = 4096;    // codes per variable-owned item (whole variables; at least one)
constexpr int kOwnVars = 1024;     // variables per variable-owned item

constexpr int align16(int x) { return (x + 15) & ~15; }

// Per-warp shared-memory staging buffer of one forward tile: clause offsets + codes.
constexpr int kFwdCtabBytes = align16((kFwdClauses + 1) * 2 + 15);
constexpr int kFwdCodeBytes = align16(kFwdCodes * 4 + 15);
constexpr int kFwdBufBytes = kFwdCtabBytes + kFwdCodeBytes;
// Per-warp staging buffer of one occurrence tile: var table + occurrence offsets + codes.
constexpr int kVarVtabBytes = align16((kVarVars + 1) * 4 + 15);
constexpr int kVarRecBytes = align16((kVarCodes + 1) * 2 + 15);
constexpr int kVarCodeBytes = align16(kVarCodes * 4 + 15);
constexpr int kVarBufBytes = kVarVtabBytes + kVarRecBytes + kVarCodeBytes;
// Two buffers (double buffering) + two mbarriers per warp.
constexpr int kFwdWarpBytes = 2 * kFwdBufBytes + 16;
constexpr int kVarWarpBytes = 2 * kVarBufBytes + 16;

constexpr int kWarps = 8;          // warps per CTA of the tiled kernels
constexpr int kThreads = kWarps * 32;

// TMA-gather variant of the variable-major pass (chunks of 32 lanes, 512-byte rows): per warp a
// ring of kRingSlots slots; a slot holds one batch of kRingBatch rows, fetched by
// kRingBatch / 4 tile::gather4 copies completing on the slot's mbarrier.
constexpr int kRingWarps = 2;
constexpr int kRingSlots = 4;
constexpr int kRingBatch = 8;
constexpr int kRowBytes = 512;
constexpr int kSlotBytes = kRingBatch * kRowBytes;
constexpr int kRingWarpBytes =
    ((kRingSlots * kSlotBytes + 2 * kVarBufBytes + 16 + kRingSlots * 8) + 127) / 128 * 128;

// ---------------------------------------------------------------------------------------------
// Clause-major literal code (forward and check tiles), one uint32 per literal occurrence:
//   bit 0     : negated literal
//   bit 1     : last literal of its clause
//   bits 2-31 : variable row (global, instance offset included)
constexpr uint32_t kFNeg = 1u, kFEnd = 2u;
constexpr int kFShift = 2;

// Variable-major occurrence code. The occurrence (t, i) of variable v in clause t at position i
// is stored as the list of the OTHER literals of clause t in clause order (positions < i, then
// positions > i), one uint32 each; its leave-one-out product is the product of their factors,
// i.e. the prefix product before i times the suffix product after i.
//   bit 0     : this other literal is negated
//   bit 1     : last code of the occurrence (the leave-one-out product is complete)
//   bit 2     : (on the last code) the occurrence's own literal is negated
//   bit 3     : (on the last code) the own literal is at position 0: this occurrence also
//               carries the clause's forward value U_t = f_i * LOO_i (each clause exactly once)
//   bits 4-31 : variable row of the other literal; kVSentinel for a unit clause (no other
//               literal, factor 1, no load)
constexpr uint32_t kVNeg = 1u, kVEnd = 2u, kVSelfNeg = 4u, kVCredit = 8u;
constexpr int kVShift = 4;
constexpr uint32_t kVSentinel = (1u << 28) - 1u;

struct FwdItem {
    int64_t code_base;   // first code of the tile in fcodes
    int64_t ctab_base;   // first entry in fctab (n_clauses + 1 uint16 offsets, relative)
    int32_t n_codes;
    int32_t n_clauses;
    int32_t inst;
    int32_t pad;
};
static_assert(sizeof(FwdItem) == 32, "FwdItem layout");

struct VarItem {
    int64_t code_base;   // first code of the tile in vcodes
    int64_t rec_base;    // first entry in vrecs (n_occ + 1 uint16 code offsets, relative)
    int64_t vtab_base;   // first entry in vtab (nv + 1 entries: occ_rel << 16 | code_rel)
    int32_t v0;          // first variable row
    int32_t nv;          // variables (1 for a part of a split variable)
    int32_t n_codes;
    int32_t n_occ;
    int32_t split;       // -1: whole variables; else the split variable's slot
    int32_t part;        // part index within the split variable
    int32_t n_parts;     // parts of the split variable
    int32_t split_row;   // first scratch row of the split variable's parts
    int32_t inst;
    int32_t kk;          // every occurrence in the tile has exactly kk codes (1..3), or 0 (mixed)
};
static_assert(sizeof(VarItem) == 64, "VarItem layout");

// Adam constants, prepared on the host in double precision.
struct AdamK {
    float step_size;      // lr / (1 - beta1^t)
    float beta1, one_minus_beta1;
    float beta2, one_minus_beta2;
    float inv_sqrt_bc2;   // 1 / sqrt(1 - beta2^t)
    float eps;
    float inv_tau;
};

// Candidate chunking of a [n][ldB] array of element size s: each lane owns VEC = 16/s
// consecutive candidates, LC lanes cover one chunk of Bc = LC * VEC candidates, and the
// G = 32 / LC lane groups of a warp work on different occurrences / clauses of the same tile.
struct Chunking {
    int vec, lc, bc, n_chunks, bpad;
};

enum Mode { kModeGrad = 0, kModeAdam = 1 };
enum Dtype { kF32 = 0, kBF16 = 1, kF16 = 2 };

struct VarParams {
    const VarItem* items;
    int32_t n_items;
    int32_t n_chunks;
    int32_t B;
    int32_t bpad;
    int64_t ldB;
    const uint32_t* codes;
    const uint16_t* recs;
    const uint32_t* vtab;
    const void* x_in;
    float* grad;             // kModeGrad
    const double* dloss;     // kModeGrad, [n_inst][B] or null
    float* delta;            // kModeAdam
    float* m;
    float* v;
    void* x_out;
    uint32_t* bits32;        // [n][2 * nwd] or null
    int32_t nwd;
    AdamK adam;
    float* loss_part;        // [n_items][bpad] or null
    float* split_part;       // [split rows][bpad]
    int32_t* split_cnt;      // [n_split][n_chunks], each cleared by the last part
    int32_t* head;
    int32_t* exit_cnt;
    int32_t* status;
    int64_t n_rows;              // variable rows (all instances): the debug build checks gathers against it
};

// Straight-through Gumbel pass (gs_st_step, Eq. 3-4 with noise): each lane owns one 32-bit word
// of the bit-packed hard assignment (32 candidates); LW lanes cover a chunk of LW words and the
// G = 32 / LW lane groups split each variable's occurrences. The integer gradient at the hard
// point is kept as a signed bit-sliced counter (kStPlanes bit planes, one bit per candidate).
constexpr int kStPlanes = 10;   // two's complement, |count| <= kVarCodes < 2^9 per tile part

struct StParams {
    const VarItem* items;
    int32_t n_items;
    int32_t n_chunks;        // chunks of LW 32-bit words
    int32_t B;
    int32_t nw32;            // 32-bit words per bits row (2 * ceil(B / 64))
    int64_t ldB;
    const uint32_t* codes;
    const uint16_t* recs;
    const uint32_t* vtab;
    const uint32_t* bits_in;     // [n][nw32] hard assignment of this step
    uint32_t* bits_out;          // [n][nw32] hard assignment of the next step
    float* delta;
    float* m;
    float* v;
    const float* noise;          // [n][ldB] logistic noise of this step, or null: generated
    const float* noise_next;     // [n][ldB] noise of the next step, or null: generated
    float* noise_out;            // [n][ldB] receives the generated next-step noise, or null
    uint64_t seed;
    int64_t step;
    AdamK adam;
    float* split_part;           // [split rows][bpad] partial integer gradients
    int32_t bpad;                // n_chunks * LW * 32
    int32_t* split_cnt;          // [n_split][n_chunks], each cleared by the last part
    int32_t* head;
    int32_t* exit_cnt;
    int32_t* status;
    int64_t n_rows;              // variable rows (all instances): the debug build checks gathers against it
};

// Candidate pool / branching selection (gs_pool_sample, gs_branch_vars).
constexpr int kPoolMaxS = 8192;   // selected rows per sample (one shared-memory sort per sample)

struct PoolParams {
    const float* delta;          // the selected candidate's logits: row v at delta[v * stride]
    int64_t stride;
    const float* noise;          // [n_rows][ldN] logistic noise of the N samples, or null: generated
    int64_t ldN;
    uint64_t seed;
    int32_t n_rows;              // rows taking part (the formula's own variables)
    int32_t N;                   // samples
    int32_t S;                   // rows selected per sample
    int32_t nw32;                // 32-bit words per bits row (2 * ceil(N / 64))
    bool branch;                 // keys from |delta| ascending (N = 1), no noise
    uint32_t* bits32;            // [n_rows][nw32] samples, or null
    uint32_t* hist;              // [N][65536]
    unsigned long long* prefix;  // [N] radix prefix (ends as the S-th largest key)
    int32_t* rem;                // [N] remaining rank
    int32_t* count;              // [N] rows appended
    int32_t* sel;                // [N][S] selected rows
    int32_t* status;
};

struct FwdParams {
    const FwdItem* items;
    int32_t n_items;
    int32_t n_chunks;
    int32_t B;
    int32_t bpad;
    int64_t ldB;
    const uint32_t* codes;
    const uint16_t* ctab;
    const void* x;
    float* loss_part;        // [n_items][bpad]
    int32_t* head;
    int32_t* exit_cnt;
    int32_t* status;
    int64_t n_rows;              // variable rows (all instances): the debug build checks gathers against it
};

struct CheckParams {
    const FwdItem* items;
    int32_t n_items;
    int32_t n_wchunks;       // word chunks of LW words
    int32_t B;
    int32_t nwd;             // uint64 words per row
    const uint32_t* codes;
    const uint16_t* ctab;
    const void* bits;        // [n][nwd] uint64 words, or [n] uint32 words (low halves) when B <= 32
    uint16_t* part16;        // [n_items][bpad16] per-tile unsat counts
    int32_t bpad16;          // nwd * 64
    int32_t* head;
    int32_t* exit_cnt;
    int32_t* status;
    int64_t n_rows;              // variable rows (all instances): the debug build checks gathers against it
};

// Work-queue control words (one int32 array per problem): heads and exit counts of the
// variable-major, forward and check queues, then the split-variable part counters. All are zero
// between launches (each kernel's last CTA rewinds its queue; the last part of a split variable
// clears its counter); gs_sync_status clears them after a timed-out launch.
constexpr int kCtlVarHead = 0, kCtlFwdHead = 1, kCtlCheckHead = 2;
constexpr int kCtlVarExit = 3, kCtlFwdExit = 4, kCtlCheckExit = 5;
constexpr int kCtlSplit = 8;

// Device status bits (sticky until read by gs_sync_status).
constexpr int32_t kStatusTimeout = 1;
constexpr int32_t kStatusSelect = 2;   // a selection found more rows than its rank (never expected)
constexpr int32_t kStatusBounds = 4;   // debug build: a gathered row index was out of range (load skipped)

// ---------------------------------------------------------------------------------------------
// Launchers (gs_kernels.cu). They return cudaGetLastError() of the launch.
cudaError_t launch_var_pass(const VarParams& p, int dtype, int mode, int lc, int grid, cudaStream_t s);
// tmap: a CUtensorMap (128 bytes) over x_in as a 2-D tensor [n rows][B columns], box {32*VEC, 1}.
cudaError_t launch_var_ring(const VarParams& p, const void* tmap, int dtype, int mode, int grid, cudaStream_t s);
// Variable pass with variable-owning lane groups (lc = 4, 8 or 16 lanes per chunk): items and
// vtab of p are the own-item table (whole variables; vtab: one {row - v0, first code, end code,
// 0} entry of 4 x uint32 per variable, in the order the lane groups take them).
cudaError_t launch_var_own(const VarParams& p, int dtype, int mode, int lc, int grid, cudaStream_t s);
int grid_var_own(int dtype, int mode, int lc);
int grid_var_ring(int dtype, int mode);
cudaError_t launch_forward(const FwdParams& p, int dtype, int lc, int grid, cudaStream_t s);
// words32: p.bits holds one uint32 word per variable (B <= 32, lw == 1).
cudaError_t launch_check(const CheckParams& p, int lw, bool words32, int grid, cudaStream_t s);
// out[v] = low 32 bits of bits[v * nwd] for v < n (the candidates 0..31 of each row).
cudaError_t launch_compact_low32(const uint64_t* bits, int64_t n, int32_t nwd, uint32_t* out, cudaStream_t s);
// Two-stage fixed-order reductions over the tiles of each instance (n_seg segments in stage 1;
// stage holds n_seg * n_inst * B values).
cudaError_t launch_loss_reduce2(const float* part, int32_t bpad, const int32_t* iptr, const int32_t* items,
                                const int64_t* n_empty, int32_t n_inst, int32_t B, int32_t n_seg, double* stage,
                                double* loss, cudaStream_t s);
cudaError_t launch_count_reduce(const uint16_t* part16, int32_t bpad16, const int32_t* iptr, const int32_t* items,
                                const int64_t* n_empty, int32_t n_inst, int32_t B, int32_t n_seg, int32_t* stage,
                                int32_t* unsat, int32_t* best, cudaStream_t s);
cudaError_t launch_st_pass(const StParams& p, int lw, int grid, cudaStream_t s);
cudaError_t launch_pool_select(const PoolParams& p, cudaStream_t s);
int grid_st_pass(int lw);
cudaError_t launch_st_noise(uint64_t seed, int64_t step, float* noise, int64_t n, int32_t B, int64_t ldB,
                            cudaStream_t s);
cudaError_t launch_st_sample(const float* delta, const float* noise, uint64_t seed, int64_t step, uint32_t* bits32,
                             int64_t n, int32_t B, int64_t ldB, int32_t nw32, cudaStream_t s);
cudaError_t launch_relax(const float* delta, void* x, int dtype, int64_t n, int32_t B, int64_t ldB,
                         float inv_tau, cudaStream_t s);
cudaError_t launch_round(const float* delta, uint32_t* bits32, int64_t n, int32_t B, int64_t ldB,
                         int32_t nwd, cudaStream_t s);
cudaError_t launch_adam(float* delta, float* m, float* v, const float* grad, void* x_out, int dtype,
                        int64_t n, int32_t B, int64_t ldB, const AdamK& k, cudaStream_t s);
cudaError_t launch_wait_selftest(int32_t* status, uint64_t limit_ns, cudaStream_t s);
// Random row gathers (gs_gather_probe): n gathers of row_bytes (16..512, a power of two) at rows
// idx[k] < n_rows of src (row stride `stride` bytes, 16-byte aligned); XOR of the data into sink.
cudaError_t launch_gather_probe(const void* src, int64_t stride, uint32_t n_rows, int32_t row_bytes,
                                const uint32_t* idx, int64_t n, uint32_t* sink, cudaStream_t s);
// Occupancy-derived persistent grid size for a tiled kernel instantiation.
int grid_var_pass(int dtype, int mode, int lc);
int grid_forward(int dtype, int lc);
int grid_check(int lw, bool words32 = false);

}  // namespace gs
