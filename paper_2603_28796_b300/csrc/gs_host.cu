// Host side of the C ABI (include/gs.h): validation, the clause->literal and var->occurrence
// tile builders, device upload, workspace, and dispatch to the kernels in gs_kernels.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "gs.h"
#include "gs_internal.h"
#include "gs_plan.h"

using namespace gs;

namespace {

thread_local std::string g_last_error;

gs_status fail(gs_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

gs_status cuda_fail(cudaError_t e, const char* what) {
    return fail(GS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// NVTX range around one entry point's host work and launches (header-only NVTX 3: without a
// profiler attached a push/pop is a check of one pointer).
struct Phase {
    explicit Phase(const char* name) { nvtxRangePushA(name); }
    ~Phase() { nvtxRangePop(); }
    Phase(const Phase&) = delete;
    Phase& operator=(const Phase&) = delete;
};

#define GS_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t e__ = (call);                            \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

template <typename T>
gs_status upload(const std::vector<T>& h, T** d, int64_t* bytes, cudaStream_t s) {
    // +64 B of zero padding: 16-byte bulk copies may round a tile's range up past the end.
    const size_t nb = h.size() * sizeof(T) + 64;
    void* p = nullptr;
    if (cudaMalloc(&p, nb) != cudaSuccess) {
        cudaGetLastError();   // an allocation failure is reported here, not by a later launch check
        return fail(GS_ERR_OOM, "cudaMalloc of index structures failed");
    }
    *d = static_cast<T*>(p);
    *bytes += static_cast<int64_t>(nb);
    GS_CUDA(cudaMemsetAsync(p, 0, nb, s), "cudaMemsetAsync");
    if (!h.empty()) GS_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
    return GS_OK;
}

// lc_max (4, 8, 16 or 32) caps the lanes per candidate chunk: smaller chunks keep a smaller
// set of relaxed-value rows resident in L2 at the price of more passes over the tiles.
Chunking chunking_for(int dtype, int32_t B, int lc_max = 32) {
    Chunking c{};
    c.vec = (dtype == kF32) ? 4 : 8;
    const int need = (B + c.vec - 1) / c.vec;
    c.lc = 4;
    while (c.lc < need && c.lc < lc_max) c.lc *= 2;
    // The variable pass writes the rounded bits as whole 32-bit words per chunk, so a chunk of
    // fewer than 32 candidates is only allowed when it is the only one.
    if (c.lc * c.vec < 32 && c.lc < need) c.lc = 32 / c.vec;
    c.bc = c.lc * c.vec;
    c.n_chunks = (B + c.bc - 1) / c.bc;
    if (c.n_chunks < 1) c.n_chunks = 1;
    c.bpad = c.n_chunks * c.bc;
    return c;
}

inline int32_t nwords(int32_t B) { return (B + 63) / 64; }

}  // namespace

// =============================================================================================
struct gs_problem {
    int device = 0;
    HostPlan h;   // statistics, offsets and per-instance lists (index arrays are released)
    int64_t device_bytes = 0;
    uint32_t* fcodes = nullptr;
    uint16_t* fctab = nullptr;
    FwdItem* fitems = nullptr;
    uint32_t* vcodes = nullptr;
    uint16_t* vrecs = nullptr;
    uint32_t* vtab = nullptr;
    VarItem* vitems = nullptr;
    int32_t* f_iptr = nullptr;
    int32_t* f_list = nullptr;
    int32_t* v_iptr = nullptr;
    int32_t* v_list = nullptr;
    uint32_t* oent = nullptr;    // variable-owned items (lane groups own whole variables)
    VarItem* oitems = nullptr;
    int32_t* o_iptr = nullptr;
    int32_t* o_list = nullptr;
    int64_t* inst_empty = nullptr;
    int32_t n_fitems = 0, n_vitems = 0, n_oitems = 0;
    int64_t n_vcodes = 0;
    int32_t* status = nullptr;   // sticky device status word
    // workspace
    int32_t* ctl = nullptr;      // [0] var head, [1] fwd head, [2] check head, [3] pad, [4..] split counters
    size_t ctl_cap = 0;          // ints
    float* part = nullptr;
    size_t part_cap = 0;         // floats
    float* split = nullptr;
    size_t split_cap = 0;
    uint64_t* bits = nullptr;
    size_t bits_cap = 0;         // words
    uint32_t* bits32c = nullptr; // low 32-bit word of each bit row (check of B <= 32)
    size_t bits32c_cap = 0;
    uint16_t* part16 = nullptr;  // per-tile unsat counts
    size_t part16_cap = 0;
    unsigned char* pool = nullptr;   // candidate-pool selection workspace
    size_t pool_cap = 0;             // bytes
    double* stage = nullptr;     // stage-1 sums of the tile reductions (double or int32)
    size_t stage_cap = 0;        // doubles
    int sms = 148;
    // tuning: caps on the lanes per candidate chunk, gather mode (gs_set_tuning)
    int var_lc_max = 32;
    int fwd_lc_max = 32;
    int var_gather = 0;
    int loss_mode = 0;
    int var_split = 0;
};

namespace {

gs_status check_device(const gs_problem* p) {
    int dev = -1;
    GS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != p->device) return fail(GS_ERR_STATE, "current CUDA device differs from the problem's device");
    return GS_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Stage-1 segments of the tile reductions: enough blocks (segments x 32-candidate slices x
// instances) to fill the GPU a few times over, but no segment shorter than 32 tiles, and at
// most 256 (a formula of 400,000 tiles and one slice gets 256 segments of ~1,600 tiles; 2,000
// tiles and 32 slices get 19). max_tiles: the largest per-instance tile count of the list.
// These are the segments of the forward tiles (clause-major loss and the exact check, whose
// final count kernel walks the segments one thread per candidate).
constexpr int32_t kMaxSegments = 256;
int32_t n_segments(const gs_problem* p, int32_t B, int32_t max_tiles) {
    const int64_t slices = static_cast<int64_t>((std::max(B, 1) + 31) / 32) * std::max(p->h.n_inst, 1);
    const int64_t fill = (4LL * p->sms + slices - 1) / slices;
    const int64_t want = std::min<int64_t>(fill, (static_cast<int64_t>(max_tiles) + 31) / 32);
    return static_cast<int32_t>(std::min<int64_t>(kMaxSegments, std::max<int64_t>(1, want)));
}
// Segments of the variable-pass loss partials (one partial per occurrence tile or owned item,
// up to a few hundred thousand per formula): the stage-1 walk is a chain of dependent loads per
// warp, so these aim at 16 blocks per SM and allow up to 1,024 segments, still no segment
// shorter than 32 tiles; the final loss kernel spreads the segments over 32 warps.
constexpr int32_t kMaxLossSegments = 1024;
int32_t n_loss_segments(const gs_problem* p, int32_t B, int32_t max_tiles) {
    const int64_t slices = static_cast<int64_t>((std::max(B, 1) + 31) / 32) * std::max(p->h.n_inst, 1);
    const int64_t fill = (16LL * p->sms + slices - 1) / slices;
    const int64_t want = std::min<int64_t>(fill, (static_cast<int64_t>(max_tiles) + 31) / 32);
    return static_cast<int32_t>(std::min<int64_t>(kMaxLossSegments, std::max<int64_t>(1, want)));
}
int32_t max_list(const std::vector<int32_t>& iptr) {
    int32_t mx = 0;
    for (size_t i = 0; i + 1 < iptr.size(); ++i) mx = std::max(mx, iptr[i + 1] - iptr[i]);
    return mx;
}

template <typename T>
gs_status grow(T** ptr, size_t* cap, size_t need, cudaStream_t s, bool in_capture, const char* what) {
    if (need <= *cap) return GS_OK;
    if (in_capture)
        return fail(GS_ERR_STATE, std::string("workspace '") + what +
                                      "' must grow during stream capture; call gs_reserve first");
    if (*ptr) {
        GS_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        cudaFree(*ptr);
        *ptr = nullptr;
        *cap = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();   // an allocation failure is reported here, not by a later launch check
        return fail(GS_ERR_OOM, std::string("workspace ") + what);
    }
    *ptr = static_cast<T*>(p);
    *cap = need;
    return GS_OK;
}

// The work-queue control words must be zero between launches (the kernels keep them so); a
// fresh allocation is cleared once.
gs_status grow_ctl(gs_problem* p, size_t need, cudaStream_t s, bool in_capture) {
    // a reallocation may return the old address, so compare capacities, not pointers
    const size_t cap_before = p->ctl_cap;
    gs_status st = grow(&p->ctl, &p->ctl_cap, need, s, in_capture, "counters");
    if (st != GS_OK) return st;
    if (p->ctl_cap != cap_before) GS_CUDA(cudaMemsetAsync(p->ctl, 0, sizeof(int32_t) * p->ctl_cap, s), "clear counters");
    return GS_OK;
}

gs_status ensure_ws(gs_problem* p, int dtype, int32_t B, bool need_bits, cudaStream_t s) {
    const bool cap = capturing(s);
    const Chunking cv = chunking_for(dtype, B, p->var_lc_max);
    const Chunking cf = chunking_for(dtype, B, p->fwd_lc_max);
    const size_t items = static_cast<size_t>(std::max(p->n_fitems, std::max(p->n_vitems, p->n_oitems)));
    const size_t bpad = static_cast<size_t>(std::max(cv.bpad, cf.bpad));
    gs_status st;
    if ((st = grow(&p->part, &p->part_cap, std::max<size_t>(1, items * bpad), s, cap, "loss partials")) != GS_OK)
        return st;
    if ((st = grow(&p->split, &p->split_cap, std::max<size_t>(1, static_cast<size_t>(p->h.n_split_rows) * cv.bpad), s,
                   cap, "split partials")) != GS_OK)
        return st;
    if ((st = grow_ctl(p, kCtlSplit + static_cast<size_t>(p->h.n_split) * cv.n_chunks, s, cap)) != GS_OK) return st;
    if (need_bits) {
        if ((st = grow(&p->bits, &p->bits_cap, std::max<size_t>(1, static_cast<size_t>(p->h.n) * nwords(B)), s, cap,
                       "bits")) != GS_OK)
            return st;
    }
    if (B <= 32 && (st = grow(&p->bits32c, &p->bits32c_cap, std::max<size_t>(1, static_cast<size_t>(p->h.n)), s, cap,
                               "compact bit rows")) != GS_OK)
        return st;
    if ((st = grow(&p->part16, &p->part16_cap,
                   std::max<size_t>(1, static_cast<size_t>(p->n_fitems) * static_cast<size_t>(nwords(B)) * 64), s, cap,
                   "check partials")) != GS_OK)
        return st;
    if ((st = grow(&p->stage, &p->stage_cap,
                   std::max<size_t>(1, static_cast<size_t>(std::max({n_segments(p, B, max_list(p->h.f_iptr)),
                                                                      n_loss_segments(p, B, max_list(p->h.v_iptr)),
                                                                      n_loss_segments(p, B, max_list(p->h.o_iptr))})) *
                                           std::max(p->h.n_inst, 1) * std::max(B, 1)),
                   s, cap, "reduction stage")) != GS_OK)
        return st;
    return GS_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

gs_status check_batch(const gs_problem* p, int dtype, int32_t B, int64_t ldB) {
    if (dtype < kF32 || dtype > kF16) return fail(GS_ERR_INVALID_ARG, "unknown dtype");
    if (B < 0 || B > (1 << 30)) return fail(GS_ERR_INVALID_ARG, "B out of range");
    if (ldB < B) return fail(GS_ERR_INVALID_ARG, "ldB < B");
    const int vec = (dtype == kF32) ? 4 : 8;
    if (ldB % vec != 0)
        return fail(GS_ERR_INVALID_ARG, "ldB must be a multiple of 4 (float) / 8 (16-bit) elements");
    if (ldB > (int64_t(1) << 30)) return fail(GS_ERR_INVALID_ARG, "ldB beyond 2^30 elements");
    if (p->h.n > 0 && ldB > (int64_t(1) << 40) / p->h.n) return fail(GS_ERR_INVALID_ARG, "ldB too large");
    return GS_OK;
}

gs_status need_ptr(const void* ptr, const char* name, bool required = true) {
    if (!ptr) return required ? fail(GS_ERR_INVALID_ARG, std::string("null ") + name) : GS_OK;
    if (!aligned16(ptr)) return fail(GS_ERR_INVALID_ARG, std::string(name) + " is not 16-byte aligned");
    return GS_OK;
}

AdamK adam_consts(const gs_adam& a, int64_t t) {
    AdamK k{};
    const double bc1 = 1.0 - std::pow(a.beta1, static_cast<double>(t));
    const double bc2 = 1.0 - std::pow(a.beta2, static_cast<double>(t));
    k.step_size = static_cast<float>(a.lr / bc1);
    k.beta1 = static_cast<float>(a.beta1);
    k.one_minus_beta1 = static_cast<float>(1.0 - a.beta1);
    k.beta2 = static_cast<float>(a.beta2);
    k.one_minus_beta2 = static_cast<float>(1.0 - a.beta2);
    k.inv_sqrt_bc2 = static_cast<float>(1.0 / std::sqrt(bc2));
    k.eps = static_cast<float>(a.eps);
    k.inv_tau = static_cast<float>(1.0 / a.tau);
    return k;
}

gs_status build(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                const int32_t* lits, HostPlan& P) {
    std::string err;
    // the caps (set by the caller in P.caps) must stay within the kernels' staging buffers
    if (P.caps.fwd_codes < 32 || P.caps.fwd_codes > kFwdCodes || P.caps.var_codes < 32 ||
        P.caps.var_codes > kVarCodes || P.caps.own_codes < 256 || P.caps.own_codes > 65536)
        return fail(GS_ERR_INVALID_ARG, "tile caps out of range (clause tiles 32..512, occurrence tiles 32..384, "
                                        "owned items 256..65536 codes)");
    const gs_status st = build_plan(n_inst, n_vars, n_clauses, clause_ptr, lits, P, &err);
    return st == GS_OK ? GS_OK : fail(st, err);
}

gs_status load(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
               const int32_t* lits, const gs_plan_opts* opts, gs_stream stream, gs_problem** out) {
    Phase phase__("gs_load");
    if (!out) return fail(GS_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    gs_problem* p = new (std::nothrow) gs_problem();
    if (!p) return fail(GS_ERR_OOM, "host allocation");
    if (opts) {
        if (opts->reserved != 0) {
            delete p;
            return fail(GS_ERR_INVALID_ARG, "gs_plan_opts.reserved must be 0");
        }
        if (opts->fwd_tile_codes) p->h.caps.fwd_codes = opts->fwd_tile_codes;
        if (opts->var_tile_codes) p->h.caps.var_codes = opts->var_tile_codes;
        if (opts->own_item_codes) p->h.caps.own_codes = opts->own_item_codes;
    }
    gs_status st = build(n_inst, n_vars, n_clauses, clause_ptr, lits, p->h);
    if (st != GS_OK) {
        delete p;
        return st;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) == cudaSuccess && sms > 0) p->sms = sms;
    HostPlan& H = p->h;
    p->n_fitems = static_cast<int32_t>(H.fitems.size());
    p->n_vitems = static_cast<int32_t>(H.vitems.size());
    p->n_oitems = static_cast<int32_t>(H.oitems.size());
    p->n_vcodes = static_cast<int64_t>(H.vcodes.size());
    int64_t& db = p->device_bytes;
    if ((st = upload(H.fcodes, &p->fcodes, &db, s)) != GS_OK || (st = upload(H.fctab, &p->fctab, &db, s)) != GS_OK ||
        (st = upload(H.fitems, &p->fitems, &db, s)) != GS_OK || (st = upload(H.vcodes, &p->vcodes, &db, s)) != GS_OK ||
        (st = upload(H.vrecs, &p->vrecs, &db, s)) != GS_OK || (st = upload(H.vtab, &p->vtab, &db, s)) != GS_OK ||
        (st = upload(H.vitems, &p->vitems, &db, s)) != GS_OK || (st = upload(H.f_iptr, &p->f_iptr, &db, s)) != GS_OK ||
        (st = upload(H.f_list, &p->f_list, &db, s)) != GS_OK || (st = upload(H.v_iptr, &p->v_iptr, &db, s)) != GS_OK ||
        (st = upload(H.v_list, &p->v_list, &db, s)) != GS_OK || (st = upload(H.oent, &p->oent, &db, s)) != GS_OK ||
        (st = upload(H.oitems, &p->oitems, &db, s)) != GS_OK || (st = upload(H.o_iptr, &p->o_iptr, &db, s)) != GS_OK ||
        (st = upload(H.o_list, &p->o_list, &db, s)) != GS_OK ||
        (st = upload(H.inst_empty, &p->inst_empty, &db, s)) != GS_OK) {
        gs_free(p);
        return st;
    }
    std::vector<int32_t> zero(1, 0);
    if ((st = upload(zero, &p->status, &db, s)) != GS_OK) {
        gs_free(p);
        return st;
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        gs_free(p);
        return cuda_fail(e, "upload synchronize");
    }
    // index arrays now live on the device only
    std::vector<uint32_t>().swap(H.fcodes);
    std::vector<uint16_t>().swap(H.fctab);
    std::vector<FwdItem>().swap(H.fitems);
    std::vector<uint32_t>().swap(H.vcodes);
    std::vector<uint16_t>().swap(H.vrecs);
    std::vector<uint32_t>().swap(H.vtab);
    std::vector<VarItem>().swap(H.vitems);
    std::vector<uint32_t>().swap(H.oent);
    std::vector<VarItem>().swap(H.oitems);
    *out = p;
    return GS_OK;
}

void fill_info(const HostPlan& H, int64_t fitems, int64_t vitems, int64_t vcodes, int64_t dev_bytes, gs_info* o) {
    std::memset(o, 0, sizeof(*o));
    o->n_vars = H.n;
    o->n_clauses = H.m;
    o->nnz = H.nnz;
    o->n_inst = H.n_inst;
    o->max_k = H.max_k;
    o->n_empty = H.n_empty;
    o->n_unit = H.n_unit;
    o->n_taut = H.n_taut;
    o->n_dup = H.n_dup;
    o->n_occ_codes = vcodes;
    o->n_fwd_tiles = fitems;
    o->n_var_tiles = vitems;
    o->n_split = H.n_split;
    o->device_bytes = dev_bytes;
    o->fwd_tile_codes = H.caps.fwd_codes;
    o->var_tile_codes = H.caps.var_codes;
    o->own_item_codes = H.caps.own_codes;
}

int lanes_for_words(int32_t nwd) {
    int lw = 1;
    while (lw < nwd && lw < 32) lw *= 2;
    return lw;
}

gs_status launch_check_all(gs_problem* p, const uint64_t* bits, int32_t B, int32_t* unsat, int32_t* best,
                           cudaStream_t s) {
    const int32_t nwd = nwords(B);
    const int lw = lanes_for_words(nwd);
    CheckParams cp{};
    cp.items = p->fitems;
    cp.n_items = p->n_fitems;
    cp.n_wchunks = (nwd + lw - 1) / lw;
    cp.B = B;
    cp.nwd = nwd;
    cp.codes = p->fcodes;
    cp.ctab = p->fctab;
    cp.bits = bits;
    cp.part16 = p->part16;
    cp.bpad16 = nwd * 64;
    cp.head = p->ctl + kCtlCheckHead;
    cp.exit_cnt = p->ctl + kCtlCheckExit;
    cp.status = p->status;
    cp.n_rows = p->h.n;
    // at most 32 candidates: gather 32-bit words from a compact copy of the rows' low halves
    const bool words32 = B <= 32 && p->bits32c != nullptr && p->bits32c_cap >= static_cast<size_t>(p->h.n);
    const int64_t total = static_cast<int64_t>(cp.n_items) * cp.n_wchunks;
    if (total > 0 && B > 0) {
        if (words32) {
            GS_CUDA(launch_compact_low32(bits, p->h.n, nwd, p->bits32c, s), "bit-row compaction launch");
            cp.bits = p->bits32c;
        }
        const int grid = static_cast<int>(std::min<int64_t>(grid_check(lw, words32), total));
        GS_CUDA(launch_check(cp, lw, words32, grid, s), "check kernel launch");
    }
    GS_CUDA(launch_count_reduce(p->part16, nwd * 64, p->f_iptr, p->f_list, p->inst_empty, p->h.n_inst, B,
                                n_segments(p, B, max_list(p->h.f_iptr)), reinterpret_cast<int32_t*>(p->stage), unsat, best,
                                s),
            "count reduce launch");
    return GS_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// Tensor map of the relaxed values x as a 2-D tensor [n rows][B columns] (row stride ldB),
// box = one row of 512 bytes (a full candidate chunk), for tile::gather4 copies.
bool encode_rows_map(CUtensorMap* tm, const void* x, int dtype, int64_t n, int32_t B, int64_t ldB) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || n <= 0 || n > 0x7fffffffLL) return false;
    const size_t es = (dtype == kF32) ? 4 : 2;
    const CUtensorMapDataType dt = (dtype == kF32)    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (dtype == kBF16) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(B), static_cast<cuuint64_t>(n)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldB) * es};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(kRowBytes / es), 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(tm, dt, 2, const_cast<void*>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Straight-through pass chunking: one 32-bit word (32 candidates) per lane, LW lanes per chunk.
struct StChunking {
    int lw, nw32, n_chunks, bpad;
};
StChunking st_chunking(int32_t B) {
    StChunking c{};
    c.nw32 = 2 * nwords(B);
    c.lw = 1;
    while (c.lw < c.nw32 && c.lw < 32) c.lw *= 2;
    c.n_chunks = std::max(1, (c.nw32 + c.lw - 1) / c.lw);
    c.bpad = c.n_chunks * c.lw * 32;
    return c;
}

gs_status ensure_st_ws(gs_problem* p, int32_t B, cudaStream_t s) {
    const bool cap = capturing(s);
    const StChunking c = st_chunking(B);
    gs_status st;
    if ((st = grow(&p->split, &p->split_cap, std::max<size_t>(1, static_cast<size_t>(p->h.n_split_rows) * c.bpad), s,
                   cap, "split partials")) != GS_OK)
        return st;
    return grow_ctl(p, kCtlSplit + static_cast<size_t>(p->h.n_split) * c.n_chunks, s, cap);
}

gs_status var_pass(gs_problem* p, int mode, const void* x_in, int dtype, int32_t B, int64_t ldB, const double* dloss,
                   float* grad, float* delta, float* m, float* v, void* x_out, const AdamK* k, double* loss,
                   uint64_t* bits, cudaStream_t s) {
    gs_status st;
    if ((st = ensure_ws(p, dtype, B, false, s)) != GS_OK) return st;
    const Chunking c = chunking_for(dtype, B, p->var_lc_max);
    VarParams vp{};
    vp.items = p->vitems;
    vp.n_items = p->n_vitems;
    vp.n_chunks = c.n_chunks;
    vp.B = B;
    vp.bpad = c.bpad;
    vp.ldB = ldB;
    vp.codes = p->vcodes;
    vp.recs = p->vrecs;
    vp.vtab = p->vtab;
    vp.x_in = x_in;
    vp.grad = grad;
    vp.dloss = dloss;
    vp.delta = delta;
    vp.m = m;
    vp.v = v;
    vp.x_out = x_out;
    vp.bits32 = reinterpret_cast<uint32_t*>(bits);
    vp.nwd = nwords(B);
    if (k) vp.adam = *k;
    vp.loss_part = loss ? p->part : nullptr;
    vp.split_part = p->split;
    vp.split_cnt = p->ctl + kCtlSplit;
    vp.head = p->ctl + kCtlVarHead;
    vp.exit_cnt = p->ctl + kCtlVarExit;
    vp.status = p->status;
    vp.n_rows = p->h.n;
    // lane groups own whole variables (var_split 2) when a chunk leaves more than one group
    const bool own = p->var_split == 2 && c.lc < 32 && p->h.own_ok;
    if (own) {
        vp.items = p->oitems;
        vp.n_items = p->n_oitems;
        vp.vtab = p->oent;
    }
    const int64_t total = static_cast<int64_t>(vp.n_items) * c.n_chunks;
    if (total > 0) {
        alignas(64) CUtensorMap tm;
        if (own) {
            const int grid = static_cast<int>(std::min<int64_t>(grid_var_own(dtype, mode, c.lc), total));
            GS_CUDA(launch_var_own(vp, dtype, mode, c.lc, grid, s), "variable pass (owned variables) launch");
        } else if (c.lc == 32 && p->var_gather == 2 && encode_rows_map(&tm, x_in, dtype, p->h.n, B, ldB)) {
            const int grid = static_cast<int>(std::min<int64_t>(grid_var_ring(dtype, mode), total));
            GS_CUDA(launch_var_ring(vp, &tm, dtype, mode, grid, s), "variable pass (TMA gather) launch");
        } else {
            const int grid = static_cast<int>(std::min<int64_t>(grid_var_pass(dtype, mode, c.lc), total));
            GS_CUDA(launch_var_pass(vp, dtype, mode, c.lc, grid, s), "variable pass launch");
        }
    }
    if (loss)
        GS_CUDA(launch_loss_reduce2(p->part, c.bpad, own ? p->o_iptr : p->v_iptr, own ? p->o_list : p->v_list,
                                    p->inst_empty, p->h.n_inst, B,
                                    n_loss_segments(p, B, max_list(own ? p->h.o_iptr : p->h.v_iptr)), p->stage, loss,
                                    s),
                "loss reduce launch");
    return GS_OK;
}

}  // namespace

// =============================================================================================
extern "C" {

void gs_adam_default(gs_adam* out) {
    if (!out) return;
    out->lr = 1.0;
    out->beta1 = 0.9;
    out->beta2 = 0.999;
    out->eps = 1e-8;
    out->tau = 1.0;
}

const char* gs_status_str(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_PARSE: return "malformed DIMACS input";
        case GS_ERR_OOM: return "out of memory";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_UNSUPPORTED: return "unsupported size";
        case GS_ERR_TIMEOUT: return "device-side wait timed out";
        case GS_ERR_STATE: return "invalid state";
    }
    return "unknown status";
}

const char* gs_last_error(void) { return g_last_error.c_str(); }

gs_status gs_inspect_cnf(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                         gs_info* out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "null out");
    HostPlan P;
    const gs_status st = build(1, &n_vars, &n_clauses, clause_ptr, lits, P);
    if (st != GS_OK) return st;
    int64_t bytes = 0;
    bytes += (P.fcodes.size() * 4 + 64) + (P.fctab.size() * 2 + 64) + (P.fitems.size() * sizeof(FwdItem) + 64);
    bytes += (P.vcodes.size() * 4 + 64) + (P.vrecs.size() * 2 + 64) + (P.vtab.size() * 4 + 64) +
             (P.vitems.size() * sizeof(VarItem) + 64);
    bytes += (P.oent.size() * 4 + 64) + (P.oitems.size() * sizeof(VarItem) + 64);
    for (const std::vector<int32_t>* l : {&P.f_iptr, &P.f_list, &P.v_iptr, &P.v_list, &P.o_iptr, &P.o_list})
        bytes += l->size() * 4 + 64;
    bytes += (P.inst_empty.size() * 8 + 64) + (4 + 64);   // + the status word
    fill_info(P, static_cast<int64_t>(P.fitems.size()), static_cast<int64_t>(P.vitems.size()),
              static_cast<int64_t>(P.vcodes.size()), bytes, out);
    return GS_OK;
}

gs_status gs_load_cnf(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                      gs_stream stream, gs_problem** out) {
    return load(1, &n_vars, &n_clauses, clause_ptr, lits, nullptr, stream, out);
}

gs_status gs_load_batch(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                        const int32_t* lits, gs_stream stream, gs_problem** out) {
    return load(n_inst, n_vars, n_clauses, clause_ptr, lits, nullptr, stream, out);
}

gs_status gs_load_batch_opts(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses,
                             const int64_t* clause_ptr, const int32_t* lits, const gs_plan_opts* opts,
                             gs_stream stream, gs_problem** out) {
    return load(n_inst, n_vars, n_clauses, clause_ptr, lits, opts, stream, out);
}

gs_status gs_load_dimacs(const char* path, gs_stream stream, gs_problem** out) {
    if (!path || !out) return fail(GS_ERR_INVALID_ARG, "null path/out");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(GS_ERR_INVALID_ARG, std::string("cannot open ") + path);
    std::string text;
    {
        char buf[1 << 16];
        size_t got;
        while ((got = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    }
    std::fclose(f);
    int64_t n = -1, m = -1;
    std::vector<int64_t> cp(1, 0);
    std::vector<int32_t> lits;
    bool header = false, open_clause = false;
    size_t pos = 0;
    const size_t len = text.size();
    while (pos < len) {
        size_t eol = text.find('\n', pos);
        if (eol == std::string::npos) eol = len;
        size_t q = pos;
        while (q < eol && (text[q] == ' ' || text[q] == '\t' || text[q] == '\r')) ++q;
        if (q == eol || text[q] == 'c' || text[q] == '%') {
            pos = eol + 1;
            continue;
        }
        const std::string ln = text.substr(q, eol - q);
        pos = eol + 1;
        if (ln[0] == 'p') {
            long long nn = -1, mm = -1;
            if (header || std::sscanf(ln.c_str(), "p cnf %lld %lld", &nn, &mm) != 2 || nn < 0 || mm < 0)
                return fail(GS_ERR_PARSE, "bad DIMACS header line");
            n = nn;
            m = mm;
            header = true;
            continue;
        }
        if (!header) return fail(GS_ERR_PARSE, "clause before the 'p cnf' header");
        const char* c = ln.c_str();
        while (*c) {
            while (*c == ' ' || *c == '\t' || *c == '\r') ++c;
            if (!*c) break;
            char* end = nullptr;
            const long long x = std::strtoll(c, &end, 10);
            if (end == c || (*end && *end != ' ' && *end != '\t' && *end != '\r'))
                return fail(GS_ERR_PARSE, std::string("unexpected token near '") + std::string(c).substr(0, 16) + "'");
            c = end;
            if (x == 0) {
                cp.push_back(static_cast<int64_t>(lits.size()));
                open_clause = false;
            } else {
                if (x > n || -x > n) return fail(GS_ERR_PARSE, "literal exceeds the header's variable count");
                lits.push_back(static_cast<int32_t>(x));
                open_clause = true;
            }
        }
    }
    if (!header) return fail(GS_ERR_PARSE, "missing 'p cnf' header");
    if (open_clause) return fail(GS_ERR_PARSE, "last clause is not terminated by 0");
    if (static_cast<int64_t>(cp.size()) - 1 != m) return fail(GS_ERR_PARSE, "clause count differs from the header");
    return gs_load_cnf(n, m, cp.data(), lits.empty() ? nullptr : lits.data(), stream, out);
}

gs_status gs_info_get(const gs_problem* p, gs_info* out) {
    if (!p || !out) return fail(GS_ERR_INVALID_ARG, "null argument");
    fill_info(p->h, p->n_fitems, p->n_vitems, p->n_vcodes, p->device_bytes, out);
    return GS_OK;
}

gs_status gs_set_tuning(gs_problem* p, const gs_tuning* t) {
    if (!p || !t) return fail(GS_ERR_INVALID_ARG, "null argument");
    auto ok = [](int32_t l) { return l == 0 || l == 4 || l == 8 || l == 16 || l == 32; };
    if (!ok(t->var_lanes) || !ok(t->fwd_lanes))
        return fail(GS_ERR_INVALID_ARG, "lanes per candidate chunk must be 0, 4, 8, 16 or 32");
    if (t->var_gather < 0 || t->var_gather > 2) return fail(GS_ERR_INVALID_ARG, "var_gather must be 0, 1 or 2");
    if (t->loss_mode < 0 || t->loss_mode > 2) return fail(GS_ERR_INVALID_ARG, "loss_mode must be 0, 1 or 2");
    if (t->var_split < 0 || t->var_split > 2) return fail(GS_ERR_INVALID_ARG, "var_split must be 0, 1 or 2");
    p->var_lc_max = t->var_lanes ? t->var_lanes : 32;
    p->fwd_lc_max = t->fwd_lanes ? t->fwd_lanes : 32;
    p->var_gather = t->var_gather;
    p->loss_mode = t->loss_mode;
    p->var_split = t->var_split;
    return GS_OK;
}

gs_status gs_get_tuning(const gs_problem* p, gs_tuning* t) {
    if (!p || !t) return fail(GS_ERR_INVALID_ARG, "null argument");
    t->var_lanes = p->var_lc_max;
    t->fwd_lanes = p->fwd_lc_max;
    t->var_gather = p->var_gather;
    t->loss_mode = p->loss_mode;
    t->var_split = p->var_split;
    return GS_OK;
}

gs_status gs_autotune(gs_problem* p, int32_t B, gs_dtype dtype, gs_stream stream, gs_tuning* out) {
    Phase phase__("gs_autotune");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st = check_device(p);
    if (st != GS_OK) return st;
    const int64_t ldB = ((static_cast<int64_t>(std::max(B, 1)) + 7) / 8) * 8;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (capturing(s)) return fail(GS_ERR_STATE, "gs_autotune cannot run during stream capture");
    const int64_t n = p->h.n;
    if (n == 0 || B == 0) {
        if (out) gs_get_tuning(p, out);
        return GS_OK;
    }
    // temporary candidate arrays: delta, m, v (float), two value buffers (dtype) and the loss
    // output, one row of B doubles per instance
    const size_t es = (static_cast<int>(dtype) == kF32) ? 4 : 2;
    const size_t fbytes = static_cast<size_t>(n) * ldB * 4, xbytes = static_cast<size_t>(n) * ldB * es;
    const size_t lbytes = static_cast<size_t>(std::max(p->h.n_inst, 1)) * static_cast<size_t>(B) * sizeof(double);
    void* mem = nullptr;
    if (cudaMalloc(&mem, 3 * fbytes + 2 * xbytes + lbytes + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(GS_ERR_OOM, "gs_autotune temporaries");
    }
    char* base = static_cast<char*>(mem);
    float* delta = reinterpret_cast<float*>(base);
    float* m = reinterpret_cast<float*>(base + fbytes);
    float* v = reinterpret_cast<float*>(base + 2 * fbytes);
    void* x0 = base + 3 * fbytes;
    void* x1 = base + 3 * fbytes + xbytes;
    double* loss = reinterpret_cast<double*>(base + 3 * fbytes + 2 * xbytes);
    auto cleanup = [&]() { cudaFree(mem); };
    // deterministic contents: delta from zeroed memory relaxes to 1/2; a few steps move it
    if (cudaMemsetAsync(mem, 0, 3 * fbytes, s) != cudaSuccess) {
        cleanup();
        return fail(GS_ERR_CUDA, "gs_autotune memset");
    }
    const gs_tuning saved{p->var_lc_max, p->fwd_lc_max, p->var_gather, p->loss_mode, p->var_split};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](auto&& fn) -> float {
        for (int i = 0; i < 2; ++i)
            if (fn() != GS_OK) return -1.0f;
        cudaEventRecord(e0, s);
        for (int i = 0; i < 3; ++i)
            if (fn() != GS_OK) return -1.0f;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / 3.0f;
    };
    int64_t step = 0;
    gs_status rs = gs_relax(p, delta, x0, dtype, B, ldB, 1.0f, stream);
    // variable-major pass: candidates per warp (lanes per chunk) x gather mode
    gs_tuning best = saved;
    float best_ms = -1.0f;
    int tried = 0;   // bit lc: effective chunk width already timed
    for (int lanes = 32; lanes >= 4 && rs == GS_OK; lanes /= 2) {
        const int lc = chunking_for(dtype, B, lanes).lc;
        if (tried & lc) continue;
        tried |= lc;
        // (gather, split): register loads with shared variables, the TMA ring (32-lane chunks),
        // variable-owning lane groups (narrower chunks)
        const int forms[3][2] = {{1, 1}, {2, 1}, {1, 2}};
        for (const auto& f : forms) {
            if (f[0] == 2 && lc != 32) continue;
            if (f[1] == 2 && (lc == 32 || !p->h.own_ok)) continue;
            p->var_lc_max = lanes;
            p->var_gather = f[0];
            p->var_split = f[1];
            if ((rs = ensure_ws(p, dtype, B, false, s)) != GS_OK) break;
            const float ms = timed([&] {
                return gs_step(p, delta, m, v, nullptr, x0, x1, dtype, B, ldB, ++step, nullptr, loss, nullptr, stream);
            });
            if (ms > 0.0f && (best_ms < 0.0f || ms < best_ms)) {
                best_ms = ms;
                best.var_lanes = lanes;
                best.var_gather = f[0];
                best.var_split = f[1];
            }
        }
    }
    // clause-major forward: lanes per chunk
    float best_f = -1.0f;
    tried = 0;
    for (int lanes = 32; lanes >= 4 && rs == GS_OK; lanes /= 2) {
        const int lc = chunking_for(dtype, B, lanes).lc;
        if (tried & lc) continue;
        tried |= lc;
        p->fwd_lc_max = lanes;
        if ((rs = ensure_ws(p, dtype, B, false, s)) != GS_OK) break;
        const float ms = timed([&] { return gs_forward(p, x0, dtype, B, ldB, loss, stream); });
        if (ms > 0.0f && (best_f < 0.0f || ms < best_f)) {
            best_f = ms;
            best.fwd_lanes = lanes;
        }
    }
    // loss inside the variable pass vs a separate forward pass, at the chosen widths
    if (rs == GS_OK) {
        p->var_lc_max = best.var_lanes;
        p->var_gather = best.var_gather;
        p->var_split = best.var_split;
        p->fwd_lc_max = best.fwd_lanes;
        float mode_ms[3] = {-1.0f, -1.0f, -1.0f};
        for (int mode = 1; mode <= 2 && rs == GS_OK; ++mode) {
            p->loss_mode = mode;
            if ((rs = ensure_ws(p, dtype, B, false, s)) != GS_OK) break;
            mode_ms[mode] = timed([&] {
                return gs_step(p, delta, m, v, nullptr, x0, x1, dtype, B, ldB, ++step, nullptr, loss, nullptr, stream);
            });
        }
        best.loss_mode = (mode_ms[2] > 0.0f && mode_ms[1] > 0.0f && mode_ms[2] < mode_ms[1]) ? 2 : 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t se = cudaStreamSynchronize(s);
    cleanup();
    p->var_lc_max = saved.var_lanes;
    p->fwd_lc_max = saved.fwd_lanes;
    p->var_gather = saved.var_gather;
    p->loss_mode = saved.loss_mode;
    p->var_split = saved.var_split;
    if (rs != GS_OK) return rs;
    if (se != cudaSuccess) return cuda_fail(se, "gs_autotune");
    if ((st = gs_set_tuning(p, &best)) != GS_OK) return st;
    if (out) *out = best;
    return gs_reserve(p, B, dtype);
}

gs_status gs_reserve(gs_problem* p, int32_t B, gs_dtype dtype) {
    Phase phase__("gs_reserve");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st = check_device(p);
    if (st != GS_OK) return st;
    if ((st = check_batch(p, dtype, B, ((B + 7) / 8) * 8)) != GS_OK) return st;
    st = ensure_ws(p, dtype, B, true, nullptr);
    if (st != GS_OK) return st;
    // First use of a kernel instantiation queries its occupancy and sets its shared-memory
    // attributes; do that here, outside any stream capture.
    const Chunking cv = chunking_for(dtype, B, p->var_lc_max);
    const Chunking cf = chunking_for(dtype, B, p->fwd_lc_max);
    grid_var_pass(dtype, kModeGrad, cv.lc);
    grid_var_pass(dtype, kModeAdam, cv.lc);
    grid_var_ring(dtype, kModeGrad);
    grid_var_ring(dtype, kModeAdam);
    if (cv.lc < 32) {
        grid_var_own(dtype, kModeGrad, cv.lc);
        grid_var_own(dtype, kModeAdam, cv.lc);
    }
    tensor_map_encoder();
    grid_forward(dtype, cf.lc);
    grid_check(lanes_for_words(nwords(B)), B <= 32);
    if (dtype == GS_F32) {
        if ((st = ensure_st_ws(p, B, nullptr)) != GS_OK) return st;
        grid_st_pass(st_chunking(B).lw);
    }
    GS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    return GS_OK;
}

gs_status gs_relax(gs_problem* p, const float* delta, void* x, gs_dtype dtype, int32_t B, int64_t ldB, float tau,
                   gs_stream stream) {
    Phase phase__("gs_relax");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    if (!(tau > 0.0f)) return fail(GS_ERR_INVALID_ARG, "tau must be > 0");
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(delta, "delta", any)) != GS_OK || (st = need_ptr(x, "x", any)) != GS_OK) return st;
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    GS_CUDA(launch_relax(delta, x, dtype, p->h.n, B, ldB, 1.0f / tau, s), "relax launch");
    return GS_OK;
}

gs_status gs_forward(gs_problem* p, const void* x, gs_dtype dtype, int32_t B, int64_t ldB, double* loss,
                     gs_stream stream) {
    Phase phase__("gs_forward");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    if ((st = need_ptr(x, "x", p->h.n > 0 && B > 0)) != GS_OK) return st;
    if (B > 0 && !loss) return fail(GS_ERR_INVALID_ARG, "null loss");
    if (loss && (reinterpret_cast<uintptr_t>(loss) & 7u)) return fail(GS_ERR_INVALID_ARG, "loss misaligned");
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (B == 0) return GS_OK;
    if ((st = ensure_ws(p, dtype, B, false, s)) != GS_OK) return st;
    const Chunking c = chunking_for(dtype, B, p->fwd_lc_max);
    FwdParams fp{};
    fp.items = p->fitems;
    fp.n_items = p->n_fitems;
    fp.n_chunks = c.n_chunks;
    fp.B = B;
    fp.bpad = c.bpad;
    fp.ldB = ldB;
    fp.codes = p->fcodes;
    fp.ctab = p->fctab;
    fp.x = x;
    fp.loss_part = p->part;
    fp.head = p->ctl + kCtlFwdHead;
    fp.exit_cnt = p->ctl + kCtlFwdExit;
    fp.status = p->status;
    fp.n_rows = p->h.n;
    const int64_t total = static_cast<int64_t>(fp.n_items) * c.n_chunks;
    if (total > 0) {
        const int grid = static_cast<int>(std::min<int64_t>(grid_forward(dtype, c.lc), total));
        GS_CUDA(launch_forward(fp, dtype, c.lc, grid, s), "forward launch");
    }
    GS_CUDA(launch_loss_reduce2(p->part, c.bpad, p->f_iptr, p->f_list, p->inst_empty, p->h.n_inst, B,
                                n_segments(p, B, max_list(p->h.f_iptr)), p->stage, loss, s),
            "loss reduce launch");
    return GS_OK;
}

gs_status gs_backward(gs_problem* p, const void* x, gs_dtype dtype, int32_t B, int64_t ldB, const double* dloss,
                      float* grad, gs_stream stream) {
    Phase phase__("gs_backward");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(x, "x", any)) != GS_OK || (st = need_ptr(grad, "grad", any)) != GS_OK) return st;
    if (dloss && (reinterpret_cast<uintptr_t>(dloss) & 7u)) return fail(GS_ERR_INVALID_ARG, "dloss misaligned");
    if ((st = check_device(p)) != GS_OK) return st;
    if (!any) return GS_OK;
    return var_pass(p, kModeGrad, x, dtype, B, ldB, dloss, grad, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, static_cast<cudaStream_t>(stream));
}

gs_status gs_step(gs_problem* p, float* delta, float* m, float* v, const float* grad, const void* x_in, void* x_out,
                  gs_dtype dtype, int32_t B, int64_t ldB, int64_t step, const gs_adam* adam, double* loss,
                  uint64_t* bits, gs_stream stream) {
    Phase phase__("gs_step");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    if (step < 1) return fail(GS_ERR_INVALID_ARG, "step must be >= 1");
    gs_adam a;
    gs_adam_default(&a);
    if (adam) a = *adam;
    if (!(a.tau > 0.0) || !(a.lr >= 0.0) || !(a.eps >= 0.0) || !(a.beta1 >= 0.0 && a.beta1 < 1.0) ||
        !(a.beta2 >= 0.0 && a.beta2 < 1.0))
        return fail(GS_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(delta, "delta", any)) != GS_OK || (st = need_ptr(m, "m", any)) != GS_OK ||
        (st = need_ptr(v, "v", any)) != GS_OK || (st = need_ptr(x_out, "x_out", false)) != GS_OK ||
        (st = need_ptr(bits, "bits", false)) != GS_OK)
        return st;
    if (grad) {
        if ((st = need_ptr(grad, "grad")) != GS_OK) return st;
        if (loss) return fail(GS_ERR_INVALID_ARG, "loss output is only produced by the fused path (grad == NULL)");
    } else {
        if ((st = need_ptr(x_in, "x_in", any)) != GS_OK) return st;
        if (!x_out && any) return fail(GS_ERR_INVALID_ARG, "the fused step (grad == NULL) needs x_out");
        if (x_in && x_in == x_out) return fail(GS_ERR_INVALID_ARG, "x_out must not alias x_in");
        if (loss && (reinterpret_cast<uintptr_t>(loss) & 7u)) return fail(GS_ERR_INVALID_ARG, "loss misaligned");
    }
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!any) return GS_OK;
    const AdamK k = adam_consts(a, step);
    if (grad) {
        GS_CUDA(launch_adam(delta, m, v, grad, x_out, dtype, p->h.n, B, ldB, k, s), "adam launch");
        if (bits)
            GS_CUDA(launch_round(delta, reinterpret_cast<uint32_t*>(bits), p->h.n, B, ldB, nwords(B), s),
                    "round launch");
        return GS_OK;
    }
    if (loss && p->loss_mode == 2) {
        // the loss at x_in from the clause-major forward pass, then the step without credits
        if ((st = gs_forward(p, x_in, dtype, B, ldB, loss, stream)) != GS_OK) return st;
        return var_pass(p, kModeAdam, x_in, dtype, B, ldB, nullptr, nullptr, delta, m, v, x_out, &k, nullptr, bits, s);
    }
    return var_pass(p, kModeAdam, x_in, dtype, B, ldB, nullptr, nullptr, delta, m, v, x_out, &k, loss, bits, s);
}

gs_status gs_round_check(gs_problem* p, const float* delta, int32_t B, int64_t ldB, uint64_t* bits, int32_t* unsat,
                         int32_t* best, gs_stream stream) {
    Phase phase__("gs_round_check");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, kF32, B, ldB)) != GS_OK) return st;
    if ((st = need_ptr(delta, "delta", p->h.n > 0 && B > 0)) != GS_OK ||
        (st = need_ptr(bits, "bits", false)) != GS_OK || (st = need_ptr(unsat, "unsat", B > 0)) != GS_OK)
        return st;
    if (best && (reinterpret_cast<uintptr_t>(best) & 3u)) return fail(GS_ERR_INVALID_ARG, "best misaligned");
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = ensure_ws(p, kF32, std::max(B, 1), bits == nullptr, s)) != GS_OK) return st;
    uint64_t* b = bits ? bits : p->bits;
    if (p->h.n > 0 && B > 0)
        GS_CUDA(launch_round(delta, reinterpret_cast<uint32_t*>(b), p->h.n, B, ldB, nwords(B), s), "round launch");
    return launch_check_all(p, b, B, unsat, best, s);
}

gs_status gs_check_bits(gs_problem* p, const uint64_t* bits, int32_t B, int32_t* unsat, int32_t* best,
                        gs_stream stream) {
    Phase phase__("gs_check_bits");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    if (B < 0 || B > (1 << 30)) return fail(GS_ERR_INVALID_ARG, "B out of range");
    gs_status st;
    if ((st = need_ptr(bits, "bits", p->h.n > 0 && B > 0)) != GS_OK || (st = need_ptr(unsat, "unsat", B > 0)) != GS_OK)
        return st;
    if (best && (reinterpret_cast<uintptr_t>(best) & 3u)) return fail(GS_ERR_INVALID_ARG, "best misaligned");
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((st = ensure_ws(p, kF32, std::max(B, 1), false, s)) != GS_OK) return st;
    return launch_check_all(p, bits, B, unsat, best, s);
}

gs_status gs_gather_probe(const void* src, int64_t n_rows, int64_t row_stride, int32_t row_bytes, const uint32_t* idx,
                          int64_t n_gathers, uint32_t* sink, gs_stream stream) {
    Phase phase__("gs_gather_probe");
    if (row_bytes < 16 || row_bytes > 512 || (row_bytes & (row_bytes - 1)))
        return fail(GS_ERR_INVALID_ARG, "row_bytes must be a power of two in 16..512");
    if (row_stride < row_bytes || (row_stride & 15)) return fail(GS_ERR_INVALID_ARG, "row_stride must be >= row_bytes and a multiple of 16");
    if (n_rows < 0 || n_rows > 0xfffffffeLL || n_gathers < 0) return fail(GS_ERR_INVALID_ARG, "sizes out of range");
    if (n_gathers > 0 && (!src || !idx || !sink)) return fail(GS_ERR_INVALID_ARG, "null pointer");
    if (src && !aligned16(src)) return fail(GS_ERR_INVALID_ARG, "src is not 16-byte aligned");
    if (idx && (reinterpret_cast<uintptr_t>(idx) & 3u)) return fail(GS_ERR_INVALID_ARG, "idx misaligned");
    if (sink && (reinterpret_cast<uintptr_t>(sink) & 3u)) return fail(GS_ERR_INVALID_ARG, "sink misaligned");
    GS_CUDA(launch_gather_probe(src, row_stride, static_cast<uint32_t>(n_rows), row_bytes, idx, n_gathers, sink,
                                static_cast<cudaStream_t>(stream)),
            "gather probe launch");
    return GS_OK;
}

gs_status gs_wait_selftest(gs_problem* p, uint32_t limit_us, gs_stream stream) {
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    if (limit_us == 0 || limit_us > 10000000u) return fail(GS_ERR_INVALID_ARG, "limit_us must be in 1..1e7");
    gs_status st = check_device(p);
    if (st != GS_OK) return st;
    GS_CUDA(launch_wait_selftest(p->status, static_cast<uint64_t>(limit_us) * 1000ull, static_cast<cudaStream_t>(stream)),
            "wait self-test launch");
    return GS_OK;
}

gs_status gs_sync_status(gs_problem* p) {
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st = check_device(p);
    if (st != GS_OK) return st;
    GS_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    int32_t h = 0;
    GS_CUDA(cudaMemcpy(&h, p->status, sizeof(h), cudaMemcpyDeviceToHost), "read status");
    if (h) {
        GS_CUDA(cudaMemset(p->status, 0, sizeof(int32_t)), "clear status");
        if (h & kStatusTimeout) {
            // a launch gave up part-way: its queue and split counters may not have been rewound
            if (p->ctl) GS_CUDA(cudaMemset(p->ctl, 0, sizeof(int32_t) * p->ctl_cap), "clear counters");
            return fail(GS_ERR_TIMEOUT, "a bounded device-side wait timed out");
        }
        if (h & kStatusSelect) return fail(GS_ERR_STATE, "a pool selection found more rows than its rank");
        if (h & kStatusBounds)
            return fail(GS_ERR_STATE, "a gathered row index was out of range (bounds-checked debug build; load skipped)");
    }
    return GS_OK;
}

void gs_free(gs_problem* p) {
    if (!p) return;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev == p->device) cudaDeviceSynchronize();
    void* ptrs[] = {p->fcodes, p->fctab,  p->fitems, p->vcodes,     p->vrecs,  p->vtab,   p->vitems,
                    p->f_iptr, p->f_list, p->v_iptr, p->v_list,     p->oent,   p->oitems, p->o_iptr,
                    p->o_list, p->status, p->ctl,    p->inst_empty, p->part,   p->split,  p->bits,
                    p->part16, p->stage,  p->pool,   p->bits32c};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

}  // extern "C"

// =============================================================================================
// Allocation-free forward (gs_forward_noalloc). The per-tile loss partials, the stage-1 sums
// of the tile reduction and the work-queue counters that gs_forward keeps in the problem's
// workspace live here in one fixed device array instead, so a call never allocates. The kernels,
// chunking and reduction order are gs_forward's, so the results are bitwise the same. The array
// is shared by every call on a device and keeps the last call's contents; the counters are
// cleared by each call and the partials and stage sums are fully rewritten before they are read.
namespace {

constexpr size_t kNoAllocHeader = 256;                     // work-queue counters (two int32)
constexpr size_t kNoAllocPartialBytes = size_t(16) << 20;  // 16 MiB of float32 tile partials
constexpr size_t kNoAllocStageBytes = size_t(4) << 20;     // 4 MiB of float64 stage-1 sums
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char
    g_noalloc_scratch[kNoAllocHeader + kNoAllocPartialBytes + kNoAllocStageBytes];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

gs_status noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kNoAllocMaxDevices) return fail(GS_ERR_UNSUPPORTED, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e, "cudaGetSymbolAddress of the no-alloc scratch");
        g_noalloc_addr[device] = ptr;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[device]);
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_forward_noalloc(gs_problem* p, const void* x, gs_dtype dtype, int32_t B, int64_t ldB,
                                        double* loss, gs_stream stream) {
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, dtype, B, ldB)) != GS_OK) return st;
    if ((st = need_ptr(x, "x", p->h.n > 0 && B > 0)) != GS_OK) return st;
    if (B > 0 && !loss) return fail(GS_ERR_INVALID_ARG, "null loss");
    if (loss && (reinterpret_cast<uintptr_t>(loss) & 7u)) return fail(GS_ERR_INVALID_ARG, "loss misaligned");
    if ((st = check_device(p)) != GS_OK) return st;
    if (B == 0) return GS_OK;
    // the same chunking (tuned lane cap) and segment count as gs_forward
    const Chunking c = chunking_for(dtype, B, p->fwd_lc_max);
    const int32_t n_seg = n_segments(p, B, max_list(p->h.f_iptr));
    const size_t need = static_cast<size_t>(p->n_fitems) * static_cast<size_t>(c.bpad) * sizeof(float);
    if (need > kNoAllocPartialBytes)
        return fail(GS_ERR_UNSUPPORTED, "gs_forward_noalloc needs " + std::to_string(need) +
                                            " bytes of tile partials (clause tiles x padded B x 4); its fixed "
                                            "scratch holds 16 MiB - use gs_forward for this size");
    const size_t need_stage = static_cast<size_t>(n_seg) * static_cast<size_t>(std::max(p->h.n_inst, 1)) *
                              static_cast<size_t>(B) * sizeof(double);
    if (need_stage > kNoAllocStageBytes)
        return fail(GS_ERR_UNSUPPORTED, "gs_forward_noalloc needs " + std::to_string(need_stage) +
                                            " bytes of stage sums (segments x instances x B x 8); its fixed "
                                            "scratch holds 4 MiB - use gs_forward for this size");
    unsigned char* base = nullptr;
    if ((st = noalloc_scratch(p->device, &base)) != GS_OK) return st;
    int32_t* head = reinterpret_cast<int32_t*>(base);
    int32_t* exit_cnt = head + 1;
    float* part = reinterpret_cast<float*>(base + kNoAllocHeader);
    double* stage = reinterpret_cast<double*>(base + kNoAllocHeader + kNoAllocPartialBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FwdParams fp{};
    fp.items = p->fitems;
    fp.n_items = p->n_fitems;
    fp.n_chunks = c.n_chunks;
    fp.B = B;
    fp.bpad = c.bpad;
    fp.ldB = ldB;
    fp.codes = p->fcodes;
    fp.ctab = p->fctab;
    fp.x = x;
    fp.loss_part = part;
    fp.head = head;
    fp.exit_cnt = exit_cnt;
    fp.status = p->status;
    fp.n_rows = p->h.n;
    GS_CUDA(cudaMemsetAsync(head, 0, 2 * sizeof(int32_t), s), "memset no-alloc counters");
    const int64_t total = static_cast<int64_t>(fp.n_items) * c.n_chunks;
    if (total > 0) {
        const int grid = static_cast<int>(std::min<int64_t>(grid_forward(dtype, c.lc), total));
        GS_CUDA(launch_forward(fp, dtype, c.lc, grid, s), "forward launch");
    }
    GS_CUDA(launch_loss_reduce2(part, c.bpad, p->f_iptr, p->f_list, p->inst_empty, p->h.n_inst, B, n_seg, stage,
                                loss, s),
            "loss reduce launch");
    return GS_OK;
}

// =============================================================================================
// Straight-through Gumbel training (Eq. 3 with noise, Eq. 4 in the forward pass).
namespace {
gs_status st_common(gs_problem* p, int32_t B, int64_t ldB) {
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = check_batch(p, kF32, B, ldB)) != GS_OK) return st;
    return GS_OK;
}
}  // namespace

gs_status gs_st_noise(gs_problem* p, uint64_t seed, int64_t step, float* noise, int32_t B, int64_t ldB,
                      gs_stream stream) {
    Phase phase__("gs_st_noise");
    gs_status st;
    if ((st = st_common(p, B, ldB)) != GS_OK) return st;
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(noise, "noise", any)) != GS_OK) return st;
    if (step < 0) return fail(GS_ERR_INVALID_ARG, "step must be >= 0");
    if ((st = check_device(p)) != GS_OK) return st;
    if (!any) return GS_OK;
    GS_CUDA(launch_st_noise(seed, step, noise, p->h.n, B, ldB, static_cast<cudaStream_t>(stream)), "noise launch");
    return GS_OK;
}

gs_status gs_st_sample(gs_problem* p, const float* delta, const float* noise, uint64_t seed, int64_t step, int32_t B,
                       int64_t ldB, uint64_t* bits, gs_stream stream) {
    Phase phase__("gs_st_sample");
    gs_status st;
    if ((st = st_common(p, B, ldB)) != GS_OK) return st;
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(delta, "delta", any)) != GS_OK || (st = need_ptr(noise, "noise", false)) != GS_OK ||
        (st = need_ptr(bits, "bits", any)) != GS_OK)
        return st;
    if (step < 0) return fail(GS_ERR_INVALID_ARG, "step must be >= 0");
    if ((st = check_device(p)) != GS_OK) return st;
    if (!any) return GS_OK;
    GS_CUDA(launch_st_sample(delta, noise, seed, step, reinterpret_cast<uint32_t*>(bits), p->h.n, B, ldB,
                             2 * nwords(B), static_cast<cudaStream_t>(stream)),
            "sample launch");
    return GS_OK;
}

gs_status gs_st_step(gs_problem* p, float* delta, float* m, float* v, const uint64_t* bits_in, uint64_t* bits_out,
                     const float* noise, const float* noise_next, float* noise_next_out, uint64_t seed, int64_t step,
                     int32_t B, int64_t ldB, const gs_adam* adam, gs_stream stream) {
    Phase phase__("gs_st_step");
    gs_status st;
    if ((st = st_common(p, B, ldB)) != GS_OK) return st;
    if (step < 1) return fail(GS_ERR_INVALID_ARG, "step must be >= 1");
    gs_adam a;
    gs_adam_default(&a);
    if (adam) a = *adam;
    if (!(a.tau > 0.0) || !(a.lr >= 0.0) || !(a.eps >= 0.0) || !(a.beta1 >= 0.0 && a.beta1 < 1.0) ||
        !(a.beta2 >= 0.0 && a.beta2 < 1.0))
        return fail(GS_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    const bool any = p->h.n > 0 && B > 0;
    if ((st = need_ptr(delta, "delta", any)) != GS_OK || (st = need_ptr(m, "m", any)) != GS_OK ||
        (st = need_ptr(v, "v", any)) != GS_OK || (st = need_ptr(bits_in, "bits_in", any)) != GS_OK ||
        (st = need_ptr(bits_out, "bits_out", any)) != GS_OK || (st = need_ptr(noise, "noise", false)) != GS_OK ||
        (st = need_ptr(noise_next, "noise_next", false)) != GS_OK ||
        (st = need_ptr(noise_next_out, "noise_next_out", false)) != GS_OK)
        return st;
    if (noise_next && noise_next_out)
        return fail(GS_ERR_INVALID_ARG, "noise_next_out is only written when noise_next is NULL (generated)");
    if (noise_next_out && (noise_next_out == noise || noise_next_out == delta || noise_next_out == m || noise_next_out == v))
        return fail(GS_ERR_INVALID_ARG, "noise_next_out must not alias noise, delta, m or v");
    if (any && static_cast<const void*>(bits_in) == static_cast<const void*>(bits_out))
        return fail(GS_ERR_INVALID_ARG, "bits_out must not alias bits_in");
    if ((st = check_device(p)) != GS_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!any) return GS_OK;
    if ((st = ensure_st_ws(p, B, s)) != GS_OK) return st;
    const StChunking c = st_chunking(B);
    StParams sp{};
    sp.items = p->vitems;
    sp.n_items = p->n_vitems;
    sp.n_chunks = c.n_chunks;
    sp.B = B;
    sp.nw32 = c.nw32;
    sp.ldB = ldB;
    sp.codes = p->vcodes;
    sp.recs = p->vrecs;
    sp.vtab = p->vtab;
    sp.bits_in = reinterpret_cast<const uint32_t*>(bits_in);
    sp.bits_out = reinterpret_cast<uint32_t*>(bits_out);
    sp.delta = delta;
    sp.m = m;
    sp.v = v;
    sp.noise = noise;
    sp.noise_next = noise_next;
    sp.noise_out = noise_next_out;
    sp.seed = seed;
    sp.step = step;
    sp.adam = adam_consts(a, step);
    sp.split_part = p->split;
    sp.bpad = c.bpad;
    sp.split_cnt = p->ctl + kCtlSplit;
    sp.head = p->ctl + kCtlVarHead;
    sp.exit_cnt = p->ctl + kCtlVarExit;
    sp.status = p->status;
    sp.n_rows = p->h.n;
    const int64_t total = static_cast<int64_t>(sp.n_items) * c.n_chunks;
    if (total > 0) {
        const int grid = static_cast<int>(std::min<int64_t>(grid_st_pass(c.lw), total));
        GS_CUDA(launch_st_pass(sp, c.lw, grid, s), "straight-through pass launch");
    }
    return GS_OK;
}

gs_status gs_tseitin3(int64_t n_vars, int64_t n_clauses, const int64_t* clause_ptr, const int32_t* lits,
                      int64_t* n_out, int64_t* m_out, int64_t* nnz_out, int64_t* clause_ptr_out, int32_t* lits_out) {
    std::string err;
    const gs_status st =
        tseitin3(n_vars, n_clauses, clause_ptr, lits, n_out, m_out, nnz_out, clause_ptr_out, lits_out, &err);
    return st == GS_OK ? GS_OK : fail(st, err);
}

// =============================================================================================
// Candidate pool and branching variables (Sec. "Partial Assignment Extraction for SAT Instances",
// Sec. "Guided Branching for UNSAT Instances").
namespace {
gs_status pool_run(gs_problem* p, const float* delta, int64_t stride, int32_t n_rows, const float* noise, int64_t ldN,
                   uint64_t seed, int32_t N, int32_t S, bool branch, uint64_t* bits, int32_t* sel, cudaStream_t s) {
    if (stride < 1) return fail(GS_ERR_INVALID_ARG, "stride must be >= 1");
    if (n_rows < 0 || n_rows > p->h.n) return fail(GS_ERR_INVALID_ARG, "n_rows outside 0..n_vars");
    if (N < 1 || N > (1 << 20)) return fail(GS_ERR_INVALID_ARG, "N outside 1..2^20");
    if (S < 1 || S > n_rows) return fail(GS_ERR_INVALID_ARG, "the selection size must be in 1..n_rows");
    if (S > kPoolMaxS) return fail(GS_ERR_UNSUPPORTED, "selection size beyond 8192 rows per sample");
    if (!delta || !sel) return fail(GS_ERR_INVALID_ARG, "null delta or selection output");
    if (noise && ldN < N) return fail(GS_ERR_INVALID_ARG, "ldN < N");
    gs_status st;
    if ((st = check_device(p)) != GS_OK) return st;
    const size_t hist_b = sizeof(uint32_t) * 65536u * static_cast<size_t>(N);
    const size_t need = hist_b + static_cast<size_t>(N) * (8 + 4 + 4) + 64;
    if ((st = grow(&p->pool, &p->pool_cap, need, s, capturing(s), "pool selection")) != GS_OK) return st;
    PoolParams pp{};
    pp.delta = delta;
    pp.stride = stride;
    pp.noise = branch ? nullptr : noise;
    pp.ldN = ldN;
    pp.seed = seed;
    pp.n_rows = n_rows;
    pp.N = N;
    pp.S = S;
    pp.nw32 = 2 * ((N + 63) / 64);
    pp.branch = branch;
    pp.bits32 = reinterpret_cast<uint32_t*>(bits);
    pp.hist = reinterpret_cast<uint32_t*>(p->pool);
    pp.prefix = reinterpret_cast<unsigned long long*>(p->pool + hist_b);
    pp.rem = reinterpret_cast<int32_t*>(p->pool + hist_b + 8 * static_cast<size_t>(N));
    pp.count = pp.rem + N;
    pp.sel = sel;
    pp.status = p->status;
    GS_CUDA(launch_pool_select(pp, s), "pool selection launch");
    return GS_OK;
}
}  // namespace

gs_status gs_pool_sample(gs_problem* p, const float* delta, int64_t stride, int32_t n_rows, const float* noise,
                         int64_t ldN, uint64_t seed, int32_t N, int32_t S, uint64_t* bits, int32_t* sel,
                         gs_stream stream) {
    Phase phase__("gs_pool_sample");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    gs_status st;
    if ((st = need_ptr(noise, "noise", false)) != GS_OK || (st = need_ptr(bits, "bits", false)) != GS_OK) return st;
    return pool_run(p, delta, stride, n_rows, noise, ldN, seed, N, S, false, bits, sel,
                    static_cast<cudaStream_t>(stream));
}

gs_status gs_branch_vars(gs_problem* p, const float* delta, int64_t stride, int32_t n_rows, int32_t d, int32_t* vars,
                         gs_stream stream) {
    Phase phase__("gs_branch_vars");
    if (!p) return fail(GS_ERR_INVALID_ARG, "null problem");
    return pool_run(p, delta, stride, n_rows, nullptr, 0, 0, 1, d, true, nullptr, vars,
                    static_cast<cudaStream_t>(stream));
}
