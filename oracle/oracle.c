/*
 * FP64 CPU oracle for the differentiable solving stage of GaloisSAT (arXiv 2603.28796).
 *
 * TEST INFRASTRUCTURE. This file is the slow, plain reference that the CUDA library is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it. It shares no code, header, table or helper with the CUDA library, and the library never
 * calls it.
 *
 * Everything is double precision, written loop by loop in the paper's order:
 *   - literal value s_i: s = x for a positive literal, s = 1 - x for a negated one (Eq. 1),
 *   - clause polynomial C_t = 1 - prod_i (1 - s_i) (Eq. 2),
 *   - loss L = - sum_t C_t (Eq. 5); the hot path minimises the equivalent
 *     L_unsat = sum_t prod_i (1 - s_i) = m + L, which has the same gradient,
 *   - relaxed variable x = y_1 = softmax over the two logits, i.e. sigma(delta / tau) with
 *     delta = theta_1 - theta_0 and no Gumbel noise (Eq. 3 with g = 0),
 *   - rounding x_hat = argmax_j y_j = [delta > 0], ties to state 0 (Eq. 4),
 *   - Adam on delta with PyTorch's defaults (Sec. "Experiment Setup": Adam, lr 0.5 on the
 *     two logits, which equals lr 1.0 on their difference).
 *
 * Candidate arrays are var-major: x[v * B + b] is variable v of candidate b.
 * Candidates are independent, so the outer loop over b runs in parallel (OpenMP); the order
 * of every sum inside one candidate is the plain order written here.
 *
 * Parity status: every function below is pinned by the tests (brute-force enumeration, the
 * paper's worked examples, finite differences, closed forms, torch autograd + torch.optim.Adam,
 * the noise generator's published known-answer vectors and the logistic law).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { O_OK = 0, O_BAD_LIT = 1, O_BAD_ARG = 2, O_NO_MEM = 3 };

int o_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int check_cnf(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits) {
    if (n < 0 || m < 0 || !clause_ptr || (m > 0 && !lits && clause_ptr[m] > 0)) return O_BAD_ARG;
    if (clause_ptr[0] != 0) return O_BAD_ARG;
    for (int64_t t = 0; t < m; t++)
        if (clause_ptr[t + 1] < clause_ptr[t]) return O_BAD_ARG;
    for (int64_t i = 0; i < clause_ptr[m]; i++) {
        const int64_t a = lits[i] < 0 ? -(int64_t)lits[i] : (int64_t)lits[i];
        if (a < 1 || a > n) return O_BAD_LIT;
    }
    return O_OK;
}

/* Literal value s (Eq. 1): x for a positive literal, 1 - x for a negated one. */
static inline double literal_value(int32_t lit, const double* x, int64_t B, int64_t b) {
    const int64_t v = (lit > 0 ? (int64_t)lit : -(int64_t)lit) - 1;
    const double xv = x[v * B + b];
    return lit > 0 ? xv : 1.0 - xv;
}

/* Neumaier's compensated summation step: (sum, comp) += y. */
static inline void neumaier_add(double* sum, double* comp, double y) {
    const double t = *sum + y;
    if (fabs(*sum) >= fabs(y))
        *comp += (*sum - t) + y;
    else
        *comp += (y - t) + *sum;
    *sum = t;
}

/* Relaxed values, Eq. 3 with g = 0 and two states: x = 1 / (1 + exp(-delta / tau)). */
int o_relax(int64_t n, int64_t B, const double* delta, double tau, double* x) {
    if (n < 0 || B < 0 || !(tau > 0.0)) return O_BAD_ARG;
    for (int64_t i = 0; i < n * B; i++) x[i] = 1.0 / (1.0 + exp(-delta[i] / tau));
    return O_OK;
}

/*
 * Forward, Eq. 2 + Eq. 5, per candidate b:
 *   unsat_loss[b] = sum_t prod_{i in t} (1 - s_i)   (L_unsat, >= 0, zero iff all C_t = 1)
 *   paper_loss[b] = - sum_t C_t,  C_t = 1 - prod_{i in t} (1 - s_i)
 * Either output may be NULL.
 */
int o_forward(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits, int64_t B,
              const double* x, double* unsat_loss, double* paper_loss) {
    const int st = check_cnf(n, m, clause_ptr, lits);
    if (st != O_OK) return st;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; b++) {
        double su = 0.0, cu = 0.0, sp = 0.0, cpp = 0.0;
        for (int64_t t = 0; t < m; t++) {
            double prod = 1.0;
            for (int64_t i = clause_ptr[t]; i < clause_ptr[t + 1]; i++)
                prod *= 1.0 - literal_value(lits[i], x, B, b);
            const double C = 1.0 - prod;
            neumaier_add(&su, &cu, prod);
            neumaier_add(&sp, &cpp, -C);
        }
        if (unsat_loss) unsat_loss[b] = su + cu;
        if (paper_loss) paper_loss[b] = sp + cpp;
    }
    return O_OK;
}

/*
 * Backward of L_unsat with respect to the relaxed values x (analytic, from Eq. 2):
 *   dL/dx_v = sum over occurrences (t, i) of v of  d(1 - s_i)/dx_v * prod_{j in t, j != i} (1 - s_j)
 * with d(1 - s_i)/dx_v = -1 for a positive literal and +1 for a negated one. The leave-one-out
 * product is a direct loop over the other literals of the clause (no division, no prefix or
 * suffix arrays), accumulated per (v, b) with compensation.
 * grad[v*B+b] receives dL/dx; scale[v*B+b] (optional) receives sum |leave-one-out product|,
 * the magnitude against which cancellation in grad is judged.
 */
int o_backward(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits, int64_t B,
               const double* x, double* grad, double* scale) {
    const int st = check_cnf(n, m, clause_ptr, lits);
    if (st != O_OK) return st;
    double* comp = (double*)calloc((size_t)(n * B > 0 ? n * B : 1), sizeof(double));
    if (!comp) return O_NO_MEM;
    for (int64_t i = 0; i < n * B; i++) {
        grad[i] = 0.0;
        if (scale) scale[i] = 0.0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; b++) {
        for (int64_t t = 0; t < m; t++) {
            const int64_t lo = clause_ptr[t], hi = clause_ptr[t + 1];
            for (int64_t i = lo; i < hi; i++) {
                double loo = 1.0;
                for (int64_t j = lo; j < hi; j++)
                    if (j != i) loo *= 1.0 - literal_value(lits[j], x, B, b);
                const int32_t li = lits[i];
                const int64_t v = (li > 0 ? (int64_t)li : -(int64_t)li) - 1;
                const double d = (li > 0) ? -1.0 : 1.0;
                neumaier_add(&grad[v * B + b], &comp[v * B + b], d * loo);
                if (scale) scale[v * B + b] += fabs(loo);
            }
        }
    }
    for (int64_t i = 0; i < n * B; i++) grad[i] += comp[i];
    free(comp);
    return O_OK;
}

/*
 * One Adam step on delta (PyTorch semantics: bias-corrected, no weight decay), given
 * gx = dL/dx at x = sigma(delta / tau):
 *   g     = gx * sigma(delta/tau) * sigma(-delta/tau) / tau      (chain rule through Eq. 3)
 *   m'    = beta1 m + (1 - beta1) g
 *   v'    = beta2 v + (1 - beta2) g^2
 *   delta'= delta - lr * (m' / (1 - beta1^t)) / (sqrt(v' / (1 - beta2^t)) + eps)
 *   x'    = sigma(delta' / tau)
 * step is 1-based. Outputs may alias inputs element-wise.
 */
int o_adam(int64_t n, int64_t B, const double* delta, const double* m, const double* v,
           const double* gx, int64_t step, double lr, double beta1, double beta2, double eps,
           double tau, double* delta_out, double* m_out, double* v_out, double* x_out) {
    if (n < 0 || B < 0 || step < 1 || !(tau > 0.0)) return O_BAD_ARG;
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n * B; i++) {
        const double z = delta[i] / tau;
        const double sig_pos = 1.0 / (1.0 + exp(-z));
        const double sig_neg = 1.0 / (1.0 + exp(z));
        const double g = gx[i] * sig_pos * sig_neg / tau;
        const double m1 = beta1 * m[i] + (1.0 - beta1) * g;
        const double v1 = beta2 * v[i] + (1.0 - beta2) * g * g;
        const double d1 = delta[i] - lr * (m1 / bc1) / (sqrt(v1 / bc2) + eps);
        m_out[i] = m1;
        v_out[i] = v1;
        delta_out[i] = d1;
        if (x_out) x_out[i] = 1.0 / (1.0 + exp(-d1 / tau));
    }
    return O_OK;
}

/*
 * Rounding (Eq. 4) and exact check: x_hat[v*B+b] = (delta > 0); unsat[b] counts the clauses
 * whose literals are all false under x_hat_b (an empty clause is always unsatisfied);
 * best = the lowest b with the minimal count (-1 when B = 0). x_hat and best may be NULL.
 */
int o_round_check(int64_t n, int64_t m, const int64_t* clause_ptr, const int32_t* lits, int64_t B,
                  const double* delta, uint8_t* x_hat, int32_t* unsat, int32_t* best) {
    const int st = check_cnf(n, m, clause_ptr, lits);
    if (st != O_OK) return st;
    uint8_t* xb = x_hat ? x_hat : (uint8_t*)malloc((size_t)(n * B > 0 ? n * B : 1));
    if (!xb) return O_NO_MEM;
    for (int64_t i = 0; i < n * B; i++) xb[i] = (delta[i] > 0.0) ? 1 : 0;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < B; b++) {
        int32_t count = 0;
        for (int64_t t = 0; t < m; t++) {
            int sat = 0;
            for (int64_t i = clause_ptr[t]; i < clause_ptr[t + 1]; i++) {
                const int32_t li = lits[i];
                const int64_t v = (li > 0 ? (int64_t)li : -(int64_t)li) - 1;
                const int xv = xb[v * B + b];
                const int lit_true = (li > 0) ? (xv == 1) : (xv == 0);
                if (lit_true) sat = 1;
            }
            if (!sat) count++;
        }
        unsat[b] = count;
    }
    if (best) {
        int32_t bi = -1;
        for (int64_t b = 0; b < B; b++)
            if (bi < 0 || unsat[b] < unsat[bi]) bi = (int32_t)b;
        *best = bi;
    }
    if (!x_hat) free(xb);
    return O_OK;
}

/*
 * ---------------------------------------------------------------------------------------------
 * Straight-through Gumbel training (Eq. 3 with noise, Eq. 4 in the forward pass).
 *
 * With two logits per variable, softmax((theta + g) / tau) puts y_1 = sigma((delta + l) / tau)
 * on state 1, delta = theta_1 - theta_0 and l = g_1 - g_0. The difference of two independent
 * Gumbel(0,1) variables is Logistic(0,1), so one logistic draw per (variable, candidate, step)
 * carries exactly the noise of Eq. 3. The forward pass uses the hard assignment
 * x_hat = argmax_j y_j = [delta + l > 0] (ties to state 0, Eq. 4); the backward pass takes the
 * gradient of the loss at x_hat and passes it through the soft y_1 (straight-through):
 *   dL/d delta = dL/dx (x_hat) * y_1 (1 - y_1) / tau.
 *
 * Noise generator (the draws are part of the method, so both sides implement one published
 * counter-based generator): Philox4x32-10 of Salmon, Moraes, Dror and Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11), with key (seed mod 2^32, seed / 2^32) and counter
 * (b / 4, row, step mod 2^32, step / 2^32); candidate b takes output word b % 4. From a 32-bit
 * word h: k = h >> 9 (23 bits), u = (k + 1/2) 2^-23 (exact in float32), l = log(u / (1 - u)).
 * ---------------------------------------------------------------------------------------------
 */
static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   /* Weyl key increments */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)M0 * x0, p1 = (uint64_t)M1 * x2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox4x32-10 block per (counter, key) pair: ctr [count][4], key [count][2], out [count][4]. */
int o_philox4x32(int64_t count, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
    if (count < 0) return O_BAD_ARG;
    for (int64_t i = 0; i < count; i++) philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
    return O_OK;
}

/*
 * Logistic noise l[v * B + b] for rows row0 .. row0 + n - 1 (row = variable row of the batch)
 * of step `step`, and optionally the 23-bit integers k it came from.
 */
int o_logistic_noise(int64_t n, int64_t B, uint64_t seed, int64_t step, int64_t row0, double* noise,
                     uint32_t* k23) {
    if (n < 0 || B < 0 || row0 < 0) return O_BAD_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; v++) {
        for (int64_t b = 0; b < B; b++) {
            const uint64_t row = (uint64_t)(row0 + v), st = (uint64_t)step;
            const uint32_t ctr[4] = {(uint32_t)(b >> 2), (uint32_t)row, (uint32_t)st, (uint32_t)(st >> 32)};
            const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
            uint32_t r[4];
            philox4x32_10(ctr, key, r);
            const uint32_t k = r[b & 3] >> 9;
            const double u = ((double)k + 0.5) / 8388608.0;   /* 2^23 */
            noise[v * B + b] = log(u / (1.0 - u));
            if (k23) k23[v * B + b] = k;
        }
    }
    return O_OK;
}

/*
 * Adam step of the straight-through Gumbel form: gx = dL/dx at the hard point x_hat, noise l of
 * the same step; z = (delta + l) / tau, y = sigma(z), g = gx * y (1 - y) / tau, then the Adam
 * update of o_adam. Outputs may alias inputs element-wise.
 */
int o_st_adam(int64_t n, int64_t B, const double* delta, const double* m, const double* v, const double* gx,
              const double* noise, int64_t step, double lr, double beta1, double beta2, double eps, double tau,
              double* delta_out, double* m_out, double* v_out) {
    if (n < 0 || B < 0 || step < 1 || !(tau > 0.0)) return O_BAD_ARG;
    const double bc1 = 1.0 - pow(beta1, (double)step);
    const double bc2 = 1.0 - pow(beta2, (double)step);
    for (int64_t i = 0; i < n * B; i++) {
        const double z = (delta[i] + noise[i]) / tau;
        const double y = 1.0 / (1.0 + exp(-z));
        const double one_minus_y = 1.0 / (1.0 + exp(z));
        const double g = gx[i] * y * one_minus_y / tau;
        const double m1 = beta1 * m[i] + (1.0 - beta1) * g;
        const double v1 = beta2 * v[i] + (1.0 - beta2) * g * g;
        m_out[i] = m1;
        v_out[i] = v1;
        delta_out[i] = delta[i] - lr * (m1 / bc1) / (sqrt(v1 / bc2) + eps);
    }
    return O_OK;
}
