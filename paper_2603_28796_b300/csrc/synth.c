/*
 * Seeded synthetic CNF generators.
 *
 * This file only produces inputs (clause widths, literal lists, a hidden planted assignment).
 * It holds none of the relaxed clause-polynomial arithmetic of the method; both the CUDA
 * library and the FP64 oracle consume what it writes.
 *
 * Randomness: xoshiro256** (Blackman & Vigna, 2018), seeded through splitmix64, written from
 * their published definitions. Every generator takes a 64-bit seed and a stream id, so that
 * widths, the hidden assignment and the literals come from independent streams.
 *
 * Literal convention: DIMACS, +(v+1) for x_v and -(v+1) for NOT x_v, 0 never appears.
 * Clause storage: CSR, clause t holds lits[clause_ptr[t] .. clause_ptr[t+1]).
 *
 * Workloads (all planted, i.e. satisfiable by construction):
 *   law 0  uniform variables (planted uniform random k-SAT),
 *   law 1  power-law variable weights w_r = (r+1)^(-1/(alpha-1)) over ranks r, ranks mapped to
 *          variables by a seeded random permutation (Chung-Lu style occurrence tail alpha),
 *   law 2  community structure: n = n_comm * S variables in contiguous blocks of S; each clause
 *          picks a home block uniformly; each literal is drawn inside the home block with
 *          probability p_in, else uniformly over all variables.
 * In every law the variables of one clause are distinct (rejection), and the signs are drawn
 * uniformly over the 2^k - 1 patterns under which the hidden assignment x* satisfies the clause.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} xo256;

static uint64_t sm64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void xo_seed(xo256* r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (0xD1B54A32D192ED03ull * (stream + 1));
    for (int i = 0; i < 4; i++) r->s[i] = sm64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo256* r) {
    uint64_t* s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* Uniform integer in [0, n), n >= 1: multiply-high with rejection of the biased low band. */
static inline uint64_t xo_below(xo256* r, uint64_t n) {
    for (;;) {
        const uint64_t x = xo_next(r);
        const __uint128_t prod = (__uint128_t)x * n;
        const uint64_t lo = (uint64_t)prod;
        if (lo >= n || lo >= (uint64_t)(-n) % n) return (uint64_t)(prod >> 64);
    }
}

/* Uniform double in [0, 1) with 53 random bits. */
static inline double xo_unit(xo256* r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

enum { SYN_OK = 0, SYN_BAD_ARG = 1, SYN_NO_MEM = 2, SYN_REJECT = 3 };

/*
 * Clause widths. law 0: every clause has width kmin. law 1: truncated geometric,
 * P(k) proportional to q^(k-kmin) on [kmin, kmax]. law 2: uniform on [kmin, kmax].
 * Writes clause_ptr[0..m] and returns nnz (or -1 on bad arguments).
 */
int64_t gs_synth_widths(uint64_t seed, int64_t m, int32_t law, int32_t kmin, int32_t kmax,
                        double q, int64_t* clause_ptr) {
    if (m < 0 || kmin < 1 || kmax < kmin || kmax > 62 || !clause_ptr) return -1;
    xo256 r;
    xo_seed(&r, seed, 1);
    double cdf[64];
    if (law == 1) {
        double acc = 0.0;
        for (int k = kmin; k <= kmax; k++) {
            acc += pow(q, (double)(k - kmin));
            cdf[k - kmin] = acc;
        }
        for (int k = kmin; k <= kmax; k++) cdf[k - kmin] /= acc;
    }
    int64_t nnz = 0;
    clause_ptr[0] = 0;
    for (int64_t t = 0; t < m; t++) {
        int k = kmin;
        if (law == 1) {
            const double u = xo_unit(&r);
            k = kmax;
            for (int j = kmin; j <= kmax; j++) {
                if (u < cdf[j - kmin]) {
                    k = j;
                    break;
                }
            }
        } else if (law == 2) {
            k = kmin + (int)xo_below(&r, (uint64_t)(kmax - kmin + 1));
        } else if (law != 0) {
            return -1;
        }
        nnz += k;
        clause_ptr[t + 1] = nnz;
    }
    return nnz;
}

/*
 * Literal lists for clause widths already in clause_ptr, planted under a hidden assignment
 * written to xstar[0..n) (0/1 bytes). law/alpha/n_comm/p_in as in the file comment.
 * Returns SYN_OK, or an error code (a clause wider than its sampling range, bad arguments).
 */
int32_t gs_synth_lits(uint64_t seed, int32_t n, int64_t m, const int64_t* clause_ptr, int32_t law,
                      double alpha, int32_t n_comm, double p_in, uint8_t* xstar, int32_t* lits) {
    if (n < 1 || m < 0 || !clause_ptr || !xstar || !lits) return SYN_BAD_ARG;
    xo256 rx, rl;
    xo_seed(&rx, seed, 2);
    xo_seed(&rl, seed, 3);
    for (int32_t v = 0; v < n; v++) xstar[v] = (uint8_t)(xo_next(&rx) >> 63);

    double* cdf = NULL;
    int32_t* perm = NULL;
    int32_t comm_size = 0;
    if (law == 1) {
        if (!(alpha > 1.0)) return SYN_BAD_ARG;
        cdf = (double*)malloc(sizeof(double) * (size_t)n);
        perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
        if (!cdf || !perm) {
            free(cdf);
            free(perm);
            return SYN_NO_MEM;
        }
        const double expo = -1.0 / (alpha - 1.0);
        double acc = 0.0;
        for (int32_t i = 0; i < n; i++) {
            acc += pow((double)i + 1.0, expo);
            cdf[i] = acc;
        }
        for (int32_t i = 0; i < n; i++) cdf[i] /= acc;
        xo256 rp;
        xo_seed(&rp, seed, 4);
        for (int32_t i = 0; i < n; i++) perm[i] = i;
        for (int32_t i = n - 1; i > 0; i--) {
            const int32_t j = (int32_t)xo_below(&rp, (uint64_t)i + 1);
            const int32_t tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
    } else if (law == 2) {
        if (n_comm < 1 || n % n_comm != 0 || p_in < 0.0 || p_in > 1.0) return SYN_BAD_ARG;
        comm_size = n / n_comm;
    } else if (law != 0) {
        return SYN_BAD_ARG;
    }

    int32_t status = SYN_OK;
    int32_t vars[64];
    for (int64_t t = 0; t < m && status == SYN_OK; t++) {
        const int64_t b = clause_ptr[t];
        const int k = (int)(clause_ptr[t + 1] - b);
        if (k < 0 || k > 62 || k > n || (law == 2 && k > comm_size)) {
            status = SYN_BAD_ARG;
            break;
        }
        const int32_t home = (law == 2) ? (int32_t)xo_below(&rl, (uint64_t)n_comm) : 0;
        for (int i = 0; i < k; i++) {
            int32_t v = 0;
            for (int attempt = 0;; attempt++) {
                if (attempt > 100000) {
                    status = SYN_REJECT;
                    break;
                }
                if (law == 0) {
                    v = (int32_t)xo_below(&rl, (uint64_t)n);
                } else if (law == 1) {
                    const double u = xo_unit(&rl);
                    int32_t lo = 0, hi = n - 1;
                    while (lo < hi) {
                        const int32_t mid = lo + (hi - lo) / 2;
                        if (u < cdf[mid])
                            hi = mid;
                        else
                            lo = mid + 1;
                    }
                    v = perm[lo];
                } else {
                    if (xo_unit(&rl) < p_in)
                        v = home * comm_size + (int32_t)xo_below(&rl, (uint64_t)comm_size);
                    else
                        v = (int32_t)xo_below(&rl, (uint64_t)n);
                }
                int dup = 0;
                for (int j = 0; j < i; j++) dup |= (vars[j] == v);
                if (!dup) break;
            }
            if (status != SYN_OK) break;
            vars[i] = v;
        }
        if (status != SYN_OK || k == 0) continue;
        /* r in [1, 2^k - 1]: bit i set <=> literal i is true under x*. */
        const uint64_t r = 1 + xo_below(&rl, (((uint64_t)1) << k) - 1);
        for (int i = 0; i < k; i++) {
            const int truth = (int)((r >> i) & 1u);
            const int positive = (truth == (int)xstar[vars[i]]);
            lits[b + i] = positive ? (vars[i] + 1) : -(vars[i] + 1);
        }
    }
    free(cdf);
    free(perm);
    return status;
}
