// Host-side tile builder: validation and statistics, the clause tiles of the forward pass and
// the check, and the occurrence tiles (the transpose) of the variable-major pass.
//
// Every stage that touches each literal runs on all host cores (contiguous blocks of clauses
// or variables per thread); the tile partition itself is a sequential sweep over per-variable
// and per-clause sizes, so the output is identical for any number of threads. Nothing inside a
// worker allocates or throws.
#include "gs_plan.h"

#include <algorithm>
#include <new>
#include <system_error>
#include <thread>

namespace gs {
namespace {

int hw_threads() {
    static const int hw = [] {
        const unsigned h = std::thread::hardware_concurrency();
        return h == 0 ? 1 : static_cast<int>(std::min(h, 64u));
    }();
    return hw;
}

// Runs f(begin, end, block) over contiguous blocks of [0, n), block b covering
// [n·b/T, n·(b+1)/T). Blocks that could not be given a thread run on the caller.
template <class F>
int parallel_blocks(int64_t n, F&& f) {
    const int T = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(hw_threads(), n / 4096)));
    auto lo = [&](int b) { return n * b / T; };
    std::vector<std::thread> th;
    int started = 1;
    try {
        th.reserve(T > 1 ? T - 1 : 0);
        for (; started < T; ++started) th.emplace_back([&f, &lo, started] { f(lo(started), lo(started + 1), started); });
    } catch (const std::exception&) {
        // fewer threads than blocks: the remaining blocks run below
    }
    f(lo(0), lo(1), 0);
    for (int b = started; b < T; ++b) f(lo(b), lo(b + 1), b);
    for (auto& t : th) t.join();
    return T;
}

inline int32_t abs32(int32_t x) { return x < 0 ? -x : x; }

// Instance owning clause t (clause_off is non-decreasing; empty instances are skipped).
inline int32_t inst_of_clause(const HostPlan& P, int64_t t) {
    return static_cast<int32_t>(std::upper_bound(P.clause_off.begin(), P.clause_off.end(), t) - P.clause_off.begin()) - 1;
}

inline int64_t lit_row(const HostPlan& P, int32_t inst, int32_t lit) {
    return P.var_off[inst] + abs32(lit) - 1;
}

// Sort of a clause's literals by (variable, sign), in place; clauses are at most 256 wide.
void sort_lits(int32_t* a, int k) {
    auto less = [](int32_t x, int32_t y) {
        const int32_t ax = abs32(x), ay = abs32(y);
        return ax != ay ? ax < ay : x < y;
    };
    if (k > 24) {
        std::sort(a, a + k, less);
        return;
    }
    for (int i = 1; i < k; ++i) {
        const int32_t x = a[i];
        int j = i - 1;
        while (j >= 0 && less(x, a[j])) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = x;
    }
}

struct BlockError {
    int64_t t = -1;   // first failing clause of the block, -1 if none
    gs_status st = GS_OK;
    int64_t a = 0, b = 0;   // details for the message
};

// Validation + statistics. Fills plan.{n, m, nnz, n_inst, max_k, stats, var_off, clause_off,
// inst_empty}.
gs_status validate(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                   const int32_t* lits, HostPlan& P, std::string* err) {
    if (n_inst < 1) return *err = "n_inst must be >= 1", GS_ERR_INVALID_ARG;
    if (!n_vars || !n_clauses || !clause_ptr) return *err = "null n_vars/n_clauses/clause_ptr", GS_ERR_INVALID_ARG;
    P.n_inst = n_inst;
    P.var_off.assign(n_inst + 1, 0);
    P.clause_off.assign(n_inst + 1, 0);
    P.inst_empty.assign(n_inst, 0);
    for (int32_t i = 0; i < n_inst; ++i) {
        if (n_vars[i] < 0 || n_clauses[i] < 0) return *err = "negative n_vars or n_clauses", GS_ERR_INVALID_ARG;
        P.var_off[i + 1] = P.var_off[i] + n_vars[i];
        P.clause_off[i + 1] = P.clause_off[i] + n_clauses[i];
        if (P.var_off[i + 1] > kMaxVars) return *err = "too many variables (limit 2^28 - 2)", GS_ERR_UNSUPPORTED;
        if (P.clause_off[i + 1] > (int64_t(1) << 40)) return *err = "too many clauses", GS_ERR_UNSUPPORTED;
    }
    P.n = P.var_off[n_inst];
    P.m = P.clause_off[n_inst];
    if (clause_ptr[0] != 0) return *err = "clause_ptr[0] must be 0", GS_ERR_INVALID_ARG;

    // pass 1: clause widths (clause_ptr non-decreasing, every width <= 256)
    std::vector<BlockError> e1(hw_threads());
    parallel_blocks(P.m, [&](int64_t t0, int64_t t1, int blk) {
        for (int64_t t = t0; t < t1; ++t) {
            const int64_t k = clause_ptr[t + 1] - clause_ptr[t];
            if (k < 0 || k > kMaxClauseWidth) {
                e1[blk] = {t, k < 0 ? GS_ERR_INVALID_ARG : GS_ERR_UNSUPPORTED, k, 0};
                return;
            }
        }
    });
    for (const BlockError& e : e1) {
        if (e.t < 0) continue;
        if (e.st == GS_ERR_INVALID_ARG) *err = "clause_ptr is decreasing at clause " + std::to_string(e.t);
        else *err = "clause " + std::to_string(e.t) + " has " + std::to_string(e.a) + " literals (limit 256)";
        return e.st;
    }
    P.nnz = clause_ptr[P.m];
    if (P.nnz > 0 && !lits) return *err = "null lits", GS_ERR_INVALID_ARG;

    // pass 2: literal ranges and statistics
    struct Stats {
        int32_t max_k = 0;
        int64_t n_empty = 0, n_unit = 0, n_dup = 0, n_taut = 0;
        BlockError e;
    };
    std::vector<Stats> st(hw_threads());
    parallel_blocks(P.m, [&](int64_t t0, int64_t t1, int blk) {
        Stats& S = st[blk];
        int32_t tmp[kMaxClauseWidth];
        int32_t inst = t0 < P.m ? inst_of_clause(P, t0) : 0;
        for (int64_t t = t0; t < t1; ++t) {
            while (t >= P.clause_off[inst + 1]) ++inst;
            const int64_t a = clause_ptr[t], b = clause_ptr[t + 1];
            const int k = static_cast<int>(b - a);
            const int64_t nv = P.var_off[inst + 1] - P.var_off[inst];
            S.max_k = std::max(S.max_k, k);
            if (k == 0) {
                S.n_empty++;
                __atomic_fetch_add(&P.inst_empty[inst], int64_t(1), __ATOMIC_RELAXED);
            }
            if (k == 1) S.n_unit++;
            for (int64_t j = a; j < b; ++j) {
                const int64_t l = lits[j];
                const int64_t av = l < 0 ? -l : l;
                if (l == 0 || av > nv) {
                    S.e = {t, GS_ERR_INVALID_ARG, l, nv};
                    return;
                }
                tmp[j - a] = lits[j];
            }
            sort_lits(tmp, k);
            bool dup = false, taut = false;
            for (int j = 1; j < k; ++j) {
                if (tmp[j] == tmp[j - 1]) dup = true;
                if (tmp[j] == -tmp[j - 1]) taut = true;
            }
            S.n_dup += dup;
            S.n_taut += taut;
        }
    });
    for (const Stats& S : st) {
        if (S.e.t >= 0) {
            *err = "literal " + std::to_string(S.e.a) + " of clause " + std::to_string(S.e.t) + " outside 1.." +
                   std::to_string(S.e.b);
            return S.e.st;
        }
    }
    for (const Stats& S : st) {
        P.max_k = std::max(P.max_k, S.max_k);
        P.n_empty += S.n_empty;
        P.n_unit += S.n_unit;
        P.n_dup += S.n_dup;
        P.n_taut += S.n_taut;
    }
    return GS_OK;
}

// Small formulas get smaller tiles so that enough warps have work: a formula of m clauses (n
// variables) is cut into at least about kMinTiles clause (occurrence) tiles when it is small
// enough, by capping the clauses (variables) per tile; large formulas hit the code limits first.
constexpr int64_t kMinTiles = 2048;
int tile_cap(int64_t count, int cap) {
    const int64_t want = (count + kMinTiles - 1) / kMinTiles;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(cap, want)));
}

// Clause tiles: whole clauses of one instance, at most caps.fwd_codes codes (<= kFwdCodes; at
// least one clause) and kFwdClauses clauses. The tiles
// take the clauses in the order of their median literal's variable row (a stable counting sort;
// an empty clause keys on its instance's first row), so that a tile's literals fall on nearby
// rows when the formula has locality (clauses of one community, chains of one long clause)
// and the rows a tile gathers stay in cache. The loss and the counts are sums over all clauses,
// so the order changes only the float32 summation order of the loss. Codes are stored in tile
// order, one per literal in literal order within each clause.
void build_fwd(const int64_t* clause_ptr, const int32_t* lits, HostPlan& P) {
    const int clause_cap = tile_cap(P.m, kFwdClauses);
    const int64_t m = P.m, n = P.n;
    // sort key of every clause: its median literal's variable row
    std::vector<int64_t> key(m);
    parallel_blocks(m, [&](int64_t t0, int64_t t1, int) {
        int32_t inst = t0 < m ? inst_of_clause(P, t0) : 0;
        std::vector<int64_t> rows;
        for (int64_t t = t0; t < t1; ++t) {
            while (t >= P.clause_off[inst + 1]) ++inst;
            const int64_t a = clause_ptr[t], b = clause_ptr[t + 1];
            if (a == b) {
                key[t] = P.var_off[inst];
                continue;
            }
            rows.clear();
            for (int64_t j = a; j < b; ++j) rows.push_back(lit_row(P, inst, lits[j]));
            std::nth_element(rows.begin(), rows.begin() + (b - a) / 2, rows.end());
            key[t] = rows[(b - a) / 2];
        }
    });
    // stable counting sort by key: instances stay contiguous and in order, since instance i's
    // rows (and the first-row key of its empty clauses) precede instance i + 1's
    std::vector<int64_t> order(m);
    {
        std::vector<int64_t> cnt(n + 2, 0);
        for (int64_t t = 0; t < m; ++t) cnt[key[t] + 1]++;
        for (int64_t r = 0; r <= n; ++r) cnt[r + 1] += cnt[r];
        for (int64_t t = 0; t < m; ++t) order[cnt[key[t]]++] = t;
    }
    std::vector<int64_t>().swap(key);
    // tiles over the sorted sequence; code offsets of the sorted clauses
    std::vector<int64_t> pos_code(m + 1, 0);
    for (int64_t i = 0; i < m; ++i) pos_code[i + 1] = pos_code[i] + (clause_ptr[order[i] + 1] - clause_ptr[order[i]]);
    std::vector<int64_t> first;   // first sorted position of each tile
    P.f_iptr.assign(P.n_inst + 1, 0);
    int64_t ctab = 0;
    for (int32_t inst = 0; inst < P.n_inst; ++inst) {
        int64_t t = P.clause_off[inst];
        const int64_t te = P.clause_off[inst + 1];
        while (t < te) {
            FwdItem it{};
            it.code_base = pos_code[t];
            it.ctab_base = ctab;
            it.inst = inst;
            first.push_back(t);
            int nc = 0, ncodes = 0;
            while (t < te && nc < clause_cap) {
                const int k = static_cast<int>(pos_code[t + 1] - pos_code[t]);
                if (nc > 0 && ncodes + k > P.caps.fwd_codes) break;
                ncodes += k;
                ++nc;
                ++t;
            }
            it.n_codes = ncodes;
            it.n_clauses = nc;
            ctab += nc + 1;
            P.fitems.push_back(it);
        }
        P.f_iptr[inst + 1] = static_cast<int32_t>(P.fitems.size());
    }
    P.fcodes.resize(P.nnz);
    P.fctab.resize(ctab);
    parallel_blocks(static_cast<int64_t>(P.fitems.size()), [&](int64_t i0, int64_t i1, int) {
        for (int64_t i = i0; i < i1; ++i) {
            const FwdItem& it = P.fitems[i];
            const int64_t t0 = first[i];
            uint16_t* tab = &P.fctab[it.ctab_base];
            uint32_t* dst = &P.fcodes[it.code_base];
            int ncodes = 0;
            for (int c = 0; c < it.n_clauses; ++c) {
                const int64_t t = order[t0 + c];
                const int64_t a = clause_ptr[t], b = clause_ptr[t + 1];
                tab[c] = static_cast<uint16_t>(ncodes);
                for (int64_t j = a; j < b; ++j) {
                    const int32_t l = lits[j];
                    uint32_t code = static_cast<uint32_t>(lit_row(P, it.inst, l)) << kFShift;
                    if (l < 0) code |= kFNeg;
                    if (j == b - 1) code |= kFEnd;
                    dst[ncodes++] = code;
                }
            }
            tab[it.n_clauses] = static_cast<uint16_t>(ncodes);
        }
    });
    P.f_list.resize(P.fitems.size());
    for (size_t i = 0; i < P.fitems.size(); ++i) P.f_list[i] = static_cast<int32_t>(i);
}

// Calls f(t, j, a, b, inst, row) for every literal j of clause t = [a, b) whose variable row
// lies in a block of rows owned by the calling thread, in clause order. Each thread scans the
// clauses of the instances overlapping its rows, so per-row state needs no atomics and each
// row's occurrences arrive in clause order.
template <class F>
void owner_scan(const HostPlan& P, const int64_t* clause_ptr, const int32_t* lits, F&& f) {
    parallel_blocks(P.n, [&](int64_t r0, int64_t r1, int) {
        if (r0 >= r1) return;
        // instances whose variable rows intersect [r0, r1)
        const int32_t i0 = static_cast<int32_t>(
            std::upper_bound(P.var_off.begin(), P.var_off.end(), r0) - P.var_off.begin() - 1);
        const int32_t i1 = static_cast<int32_t>(
            std::lower_bound(P.var_off.begin(), P.var_off.end(), r1) - P.var_off.begin());
        for (int32_t inst = i0; inst < i1 && inst < P.n_inst; ++inst) {
            const int64_t base = P.var_off[inst] - 1;
            for (int64_t t = P.clause_off[inst]; t < P.clause_off[inst + 1]; ++t) {
                const int64_t a = clause_ptr[t], b = clause_ptr[t + 1];
                for (int64_t j = a; j < b; ++j) {
                    const int64_t row = base + abs32(lits[j]);
                    if (row >= r0 && row < r1) f(t, j, a, b, inst, row);
                }
            }
        }
    });
}

// Occurrence tiles: the transpose of the clause CSR. Occurrence (t, i) of variable v emits the
// other literals of clause t in clause order (prefix then suffix of position i); a variable's
// occurrences are listed in clause order and its codes are contiguous, variables in row order.
// The last code of every occurrence carries kVEnd, so occurrence boundaries are recovered from
// the codes themselves when the tiles' offset tables are filled.
gs_status build_var(const int64_t* clause_ptr, const int32_t* lits, HostPlan& P) {
    const int64_t n = P.n;
    auto width = [](int64_t k) -> int { return k > 1 ? static_cast<int>(k - 1) : 1; };
    auto combine_kk = [](int acc, int k) { return acc == -1 ? k : (acc == k ? acc : 0); };
    // per-variable occurrences and codes (clause-parallel counting)
    std::vector<int64_t> occ_cnt(n, 0), code_pos(n + 1, 0);
    parallel_blocks(P.m, [&](int64_t t0, int64_t t1, int) {
        int32_t inst = t0 < P.m ? inst_of_clause(P, t0) : 0;
        for (int64_t t = t0; t < t1; ++t) {
            while (t >= P.clause_off[inst + 1]) ++inst;
            const int64_t a = clause_ptr[t], b = clause_ptr[t + 1];
            const int64_t w = width(b - a);
            for (int64_t j = a; j < b; ++j) {
                const int64_t row = lit_row(P, inst, lits[j]);
                __atomic_fetch_add(&occ_cnt[row], int64_t(1), __ATOMIC_RELAXED);
                __atomic_fetch_add(&code_pos[row + 1], w, __ATOMIC_RELAXED);
            }
        }
    });
    for (int64_t v = 0; v < n; ++v) code_pos[v + 1] += code_pos[v];
    std::vector<int64_t> code_start(code_pos.begin(), code_pos.end());
    auto cost = [&](int64_t v) { return code_start[v + 1] - code_start[v]; };
    // codes, scattered straight from the clause scan
    P.vcodes.resize(code_start[n]);
    owner_scan(P, clause_ptr, lits, [&](int64_t, int64_t j, int64_t a, int64_t b, int32_t inst, int64_t row) {
        uint32_t* dst = P.vcodes.data() + code_pos[row];
        const int32_t own = lits[j];
        uint32_t tail = kVEnd;
        if (own < 0) tail |= kVSelfNeg;
        if (j == a) tail |= kVCredit;
        if (b - a == 1) {
            dst[0] = (kVSentinel << kVShift) | tail;
            code_pos[row] += 1;
            return;
        }
        const int64_t last = (j == b - 1) ? b - 2 : b - 1;
        int c = 0;
        for (int64_t q = a; q < b; ++q) {
            if (q == j) continue;
            const int32_t l = lits[q];
            uint32_t code = static_cast<uint32_t>(lit_row(P, inst, l)) << kVShift;
            if (l < 0) code |= kVNeg;
            if (q == last) code |= tail;
            dst[c++] = code;
        }
        code_pos[row] += c;
    });
    std::vector<int64_t>().swap(code_pos);
    // Each variable's credited occurrences (the clause's loss credit sits at this literal) are
    // moved to the front of its list, keeping the clause order within both parts; credit_len is
    // the credited part's code count. The owned-variable pass runs the credit arithmetic only
    // over that part (the fourth field of its item entries marks where it ends).
    std::vector<int64_t> credit_len(n, 0);
    parallel_blocks(n, [&](int64_t v0, int64_t v1, int) {
        std::vector<uint32_t> tmp;
        for (int64_t v = v0; v < v1; ++v) {
            uint32_t* c = P.vcodes.data() + code_start[v];
            const int64_t len = code_start[v + 1] - code_start[v];
            tmp.assign(c, c + len);
            int64_t out = 0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int64_t q = 0; q < len;) {
                    int64_t e = q;
                    while (!(tmp[e] & kVEnd)) ++e;
                    const bool credited = (tmp[e] & kVCredit) != 0u;
                    if (credited == (pass == 0))
                        for (int64_t r = q; r <= e; ++r) c[out++] = tmp[r];
                    q = e + 1;
                }
                if (pass == 0) credit_len[v] = out;
            }
        }
    });
    const uint32_t* codes = P.vcodes.data();

    // Sequential partition into tiles (creation order = storage order of recs and vtab).
    const int var_cap = tile_cap(n, kVarVars);
    struct Pending {
        size_t made;
        int64_t cost;     // codes of the whole split variable (ordering key)
    };
    std::vector<VarItem> made;
    std::vector<Pending> split;
    int64_t recs = 0, vtab = 0;
    for (int32_t inst = 0; inst < P.n_inst; ++inst) {
        const int64_t ra = P.var_off[inst], rb = P.var_off[inst + 1];
        VarItem cur{};
        bool open = false;
        auto close_item = [&]() {
            if (!open) return;
            vtab += 1;
            recs += 1;
            made.push_back(cur);
            open = false;
        };
        for (int64_t v = ra; v < rb; ++v) {
            if (cost(v) > P.caps.var_codes) {
                close_item();
                // parts of <= var_codes codes (at least one occurrence), split at occurrence
                // boundaries
                const int32_t slot = P.n_split++;
                const int32_t row0 = P.n_split_rows;
                const size_t first_part = made.size();
                int64_t q = code_start[v];
                const int64_t qe = code_start[v + 1];
                int32_t pi = 0;
                while (q < qe) {
                    VarItem it{};
                    it.code_base = q;
                    it.rec_base = recs;
                    it.vtab_base = vtab;
                    it.v0 = static_cast<int32_t>(v);
                    it.nv = 1;
                    it.split = slot;
                    it.part = pi++;
                    it.split_row = row0;
                    it.inst = inst;
                    int c = 0, kk = -1;
                    while (q < qe) {
                        int w = 1;
                        while (!(codes[q + w - 1] & kVEnd)) ++w;   // this occurrence's codes
                        if (c > 0 && c + w > P.caps.var_codes) break;
                        c += w;
                        q += w;
                        kk = combine_kk(kk, w);
                        it.n_occ++;
                    }
                    it.n_codes = c;
                    it.kk = (kk >= 1 && kk <= 3) ? kk : 0;
                    recs += it.n_occ + 1;
                    vtab += 2;
                    made.push_back(it);
                }
                for (size_t k = first_part; k < made.size(); ++k) {
                    made[k].n_parts = pi;
                    split.push_back({k, cost(v)});
                }
                P.n_split_rows += pi;
                continue;
            }
            if (open && (cur.nv == var_cap || cur.n_codes + cost(v) > P.caps.var_codes)) close_item();
            if (!open) {
                cur = VarItem{};
                cur.code_base = code_start[v];
                cur.rec_base = recs;
                cur.vtab_base = vtab;
                cur.v0 = static_cast<int32_t>(v);
                cur.split = -1;
                cur.inst = inst;
                open = true;
            }
            vtab += 1;
            recs += occ_cnt[v];
            cur.n_occ += static_cast<int32_t>(occ_cnt[v]);
            cur.n_codes += static_cast<int32_t>(cost(v));
            cur.nv++;
        }
        close_item();
    }

    // Offset tables of every tile, from the occurrence boundaries in its codes; the uniform
    // occurrence width of whole-variable tiles.
    P.vrecs.resize(recs);
    P.vtab.resize(vtab);
    parallel_blocks(static_cast<int64_t>(made.size()), [&](int64_t i0, int64_t i1, int) {
        for (int64_t i = i0; i < i1; ++i) {
            VarItem& it = made[i];
            const uint32_t* src = codes + it.code_base;
            uint16_t* rec = P.vrecs.data() + it.rec_base;
            uint32_t* tab = P.vtab.data() + it.vtab_base;
            int32_t occ_rel = 0, code_rel = 0;
            int kk = -1;
            auto occurrences = [&](int64_t count) {
                for (int64_t o = 0; o < count; ++o) {
                    *rec++ = static_cast<uint16_t>(code_rel);
                    const int32_t c0 = code_rel;
                    while (!(src[code_rel] & kVEnd)) ++code_rel;
                    ++code_rel;
                    ++occ_rel;
                    kk = combine_kk(kk, code_rel - c0);
                }
            };
            if (it.split >= 0) {
                *tab++ = 0u;
                occurrences(it.n_occ);
            } else {
                for (int64_t v = it.v0; v < it.v0 + it.nv; ++v) {
                    *tab++ = (static_cast<uint32_t>(occ_rel) << 16) | static_cast<uint32_t>(code_rel);
                    occurrences(occ_cnt[v]);
                }
                it.kk = (kk >= 1 && kk <= 3) ? kk : 0;
            }
            *rec = static_cast<uint16_t>(code_rel);
            *tab = (static_cast<uint32_t>(occ_rel) << 16) | static_cast<uint32_t>(code_rel);
        }
    });

    // Schedule: parts of split variables first, largest variable first (they finish last
    // otherwise), then whole-variable tiles in variable order.
    std::stable_sort(split.begin(), split.end(), [](const Pending& a, const Pending& b) { return a.cost > b.cost; });
    P.vitems.clear();
    P.vitems.reserve(made.size());
    for (const Pending& s : split) P.vitems.push_back(made[s.made]);
    for (const VarItem& it : made)
        if (it.split < 0) P.vitems.push_back(it);
    // per-instance lists, ascending tile id
    std::vector<int32_t> cnt(P.n_inst + 1, 0);
    for (const VarItem& it : P.vitems) cnt[it.inst + 1]++;
    for (int32_t i = 0; i < P.n_inst; ++i) cnt[i + 1] += cnt[i];
    P.v_iptr = cnt;
    P.v_list.resize(P.vitems.size());
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k < P.vitems.size(); ++k) P.v_list[fill[P.vitems[k].inst]++] = static_cast<int32_t>(k);

    // Variable-owned items: consecutive whole variables of one instance, closed at a multiple of
    // 8 variables once they hold own_cap codes (or at kOwnVars variables, or the instance's end).
    // Within an item the variables are listed in the order the lane groups take them: by code
    // count, largest first (ties by row), so that the G groups, which take every G-th entry,
    // work on variables of similar size at the same time.
    std::vector<int32_t> vk(n, -1);   // codes per occurrence of v if all equal, 0 mixed, -1 none
    parallel_blocks(n, [&](int64_t v0, int64_t v1, int) {
        for (int64_t v = v0; v < v1; ++v) {
            int kk = -1;
            for (int64_t q = code_start[v]; q < code_start[v + 1];) {
                const int64_t q0 = q;
                while (!(codes[q] & kVEnd)) ++q;
                ++q;
                kk = combine_kk(kk, static_cast<int>(q - q0));
            }
            vk[v] = kk;
        }
    });
    const int64_t own_cap =
        std::max<int64_t>(256, std::min<int64_t>(P.caps.own_codes, code_start[n] / kMinTiles));
    P.oitems.clear();
    P.oent.clear();
    std::vector<int32_t> order;
    for (int32_t inst = 0; inst < P.n_inst; ++inst) {
        VarItem cur{};
        int kk = -1;
        bool open = false;
        auto close_own = [&]() {
            if (!open) return;
            order.resize(cur.nv);
            for (int32_t i = 0; i < cur.nv; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(),
                             [&](int32_t a, int32_t b) { return cost(cur.v0 + a) > cost(cur.v0 + b); });
            for (int32_t i : order) {
                const int64_t v = cur.v0 + i;
                P.oent.push_back(static_cast<uint32_t>(i));
                P.oent.push_back(static_cast<uint32_t>(code_start[v] - cur.code_base));
                P.oent.push_back(static_cast<uint32_t>(code_start[v + 1] - cur.code_base));
                P.oent.push_back(static_cast<uint32_t>(code_start[v] + credit_len[v] - cur.code_base));
            }
            cur.kk = (kk >= 1 && kk <= 3) ? kk : 0;
            P.oitems.push_back(cur);
            open = false;
        };
        for (int64_t v = P.var_off[inst]; v < P.var_off[inst + 1]; ++v) {
            if (!open) {
                cur = VarItem{};
                cur.code_base = code_start[v];
                cur.vtab_base = static_cast<int64_t>(P.oent.size() / 4);
                cur.v0 = static_cast<int32_t>(v);
                cur.split = -1;
                cur.inst = inst;
                kk = -1;
                open = true;
            }
            if (cost(v) > (int64_t(1) << 30)) P.own_ok = false;
            cur.nv++;
            cur.n_codes += static_cast<int32_t>(cost(v));
            if (vk[v] != -1) kk = combine_kk(kk, vk[v]);
            if ((cur.n_codes >= own_cap && cur.nv % 8 == 0) || cur.nv >= kOwnVars) close_own();
        }
        close_own();
    }
    std::fill(cnt.begin(), cnt.end(), 0);
    for (const VarItem& it : P.oitems) cnt[it.inst + 1]++;
    for (int32_t i = 0; i < P.n_inst; ++i) cnt[i + 1] += cnt[i];
    P.o_iptr = cnt;
    P.o_list.resize(P.oitems.size());
    std::vector<int32_t> ofill(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k < P.oitems.size(); ++k) P.o_list[ofill[P.oitems[k].inst]++] = static_cast<int32_t>(k);
    return GS_OK;
}

}  // namespace

gs_status build_plan(int32_t n_inst, const int64_t* n_vars, const int64_t* n_clauses, const int64_t* clause_ptr,
                     const int32_t* lits, HostPlan& P, std::string* err) {
    try {
        gs_status st = validate(n_inst, n_vars, n_clauses, clause_ptr, lits, P, err);
        if (st != GS_OK) return st;
        build_fwd(clause_ptr, lits, P);
        return build_var(clause_ptr, lits, P);
    } catch (const std::bad_alloc&) {
        *err = "host allocation failed while building tiles";
        return GS_ERR_OOM;
    } catch (const std::system_error& e) {
        *err = std::string("host thread error while building tiles: ") + e.what();
        return GS_ERR_OOM;
    }
}

gs_status tseitin3(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits, int64_t* n_out,
                   int64_t* m_out, int64_t* nnz_out, int64_t* cp_out, int32_t* lits_out, std::string* err) {
    if (!n_out || !m_out || !nnz_out) return *err = "null size output", GS_ERR_INVALID_ARG;
    HostPlan P;
    gs_status st;
    try {
        st = validate(1, &n, &m, clause_ptr, lits, P, err);
    } catch (const std::bad_alloc&) {
        return *err = "host allocation failed", GS_ERR_OOM;
    }
    if (st != GS_OK) return st;
    int64_t n2 = n, m2 = 0, nnz2 = 0;
    for (int64_t t = 0; t < m; ++t) {
        const int64_t u = clause_ptr[t + 1] - clause_ptr[t];
        if (u == 0) {
            m2 += 1;
        } else if (u <= 3) {
            m2 += 1;
            nnz2 += 3;
        } else {
            m2 += u - 2;
            nnz2 += 3 * (u - 2);
            n2 += u - 3;
        }
    }
    if (n2 > kMaxVars) return *err = "normalised formula has too many variables (limit 2^28 - 2)", GS_ERR_UNSUPPORTED;
    *n_out = n2;
    *m_out = m2;
    *nnz_out = nnz2;
    if (!cp_out && !lits_out) return GS_OK;
    if (!cp_out || !lits_out) return *err = "cp_out and lits_out must both be given", GS_ERR_INVALID_ARG;
    int64_t c = 0, j = 0;
    int32_t fresh = static_cast<int32_t>(n);   // last variable number used
    cp_out[0] = 0;
    auto emit = [&](int32_t a, int32_t b, int32_t d) {
        lits_out[j++] = a;
        lits_out[j++] = b;
        lits_out[j++] = d;
        cp_out[++c] = j;
    };
    for (int64_t t = 0; t < m; ++t) {
        const int32_t* l = lits + clause_ptr[t];
        const int64_t u = clause_ptr[t + 1] - clause_ptr[t];
        if (u == 0) {
            cp_out[++c] = j;
        } else if (u == 1) {
            emit(l[0], l[0], l[0]);
        } else if (u == 2) {
            emit(l[0], l[1], l[1]);
        } else if (u == 3) {
            emit(l[0], l[1], l[2]);
        } else {
            int32_t f = ++fresh;
            emit(l[0], l[1], f);
            for (int64_t i = 2; i < u - 2; ++i) {
                const int32_t g = ++fresh;
                emit(-f, l[i], g);
                f = g;
            }
            emit(-f, l[u - 2], l[u - 1]);
        }
    }
    return GS_OK;
}

}  // namespace gs
