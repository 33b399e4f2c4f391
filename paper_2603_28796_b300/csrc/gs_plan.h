// Host image of the device index structures and its builder (gs_plan.cpp). Internal to the
// library; the layout of each array is described in gs_internal.h.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "gs.h"
#include "gs_internal.h"

namespace gs {

// Tile size caps of the builder (gs_plan_opts); each at most the compile-time buffer size of its
// tile kind. A tile always takes at least one whole clause (occurrence), which fits any cap's
// buffer since a clause has at most kMaxClauseWidth literals.
struct PlanCaps {
    int fwd_codes = kFwdCodes;     // literal codes per clause tile
    int var_codes = kVarCodes;     // occurrence codes per occurrence tile (or split part)
    int own_codes = kOwnCodes;     // codes per owned-variable item (target)
};

struct HostPlan {
    PlanCaps caps;
    int64_t n = 0, m = 0, nnz = 0;
    int32_t n_inst = 0, max_k = 0;
    int64_t n_empty = 0, n_unit = 0, n_taut = 0, n_dup = 0;
    std::vector<int64_t> var_off, clause_off, inst_empty;
    // clause tiles
    std::vector<uint32_t> fcodes;
    std::vector<uint16_t> fctab;
    std::vector<FwdItem> fitems;
    // occurrence tiles
    std::vector<uint32_t> vcodes;
    std::vector<uint16_t> vrecs;
    std::vector<uint32_t> vtab;
    std::vector<VarItem> vitems;
    int32_t n_split = 0, n_split_rows = 0;
    // variable-owned items: runs of whole variables (codes shared with the occurrence tiles);
    // oent holds one 4 x uint32 entry per variable {row - v0, first code, end code, end of the
    // credited occurrences' codes} (codes relative to the item's first code) in the order the
    // lane groups take them
    std::vector<uint32_t> oent;
    std::vector<VarItem> oitems;
    bool own_ok = true;   // false if a variable has too many codes for an item's 32-bit counts
    // per-instance tile lists (ascending tile ids)
    std::vector<int32_t> f_iptr, f_list, v_iptr, v_list, o_iptr, o_list;
};

// Validates a batch of formulas (instance-concatenated clause CSR, DIMACS literals local to
// their instance) and builds the clause tiles and the occurrence tiles. The result depends only
// on the input, never on the number of threads used. On failure returns the status and sets
// *err to a one-line reason; P is then unspecified.
gs_status build_plan(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                     const int32_t* lits, HostPlan& P, std::string* err);

// Chain (Tseitin) normalisation to width 3 (Sec. "Clause Normalization for Vectorization", Eq. 6-8):
// a clause of u > 3 literals becomes (l1 v l2 v f1) (-f1 v l3 v f2) ... (-f_{u-3} v l_{u-1} v l_u)
// with fresh variables f numbered after the formula's own (in clause order); a clause of u = 1 or
// 2 literals repeats its last literal up to 3; u = 3 is kept; an empty clause stays empty.
// With cp_out / lits_out NULL only the sizes are returned. Errors as build_plan's validation.
gs_status tseitin3(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits, int64_t* n_out,
                   int64_t* m_out, int64_t* nnz_out, int64_t* cp_out, int32_t* lits_out, std::string* err);

}  // namespace gs
