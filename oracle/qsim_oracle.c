/*
 * qsim_oracle.c -- plain, slow CPU oracle for reversible wiring-diagram
 * simulation (J. R. Burger, "New approaches to quantum computer simulation
 * in a classical supercomputer").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this file: it exists so that tests, the smoke check and the
 * benchmark's CPU-baseline leg can compare the CUDA library against an
 * independent restatement of the paper.  It shares no header, helper or
 * table with the CUDA sources; the step record below has the same byte
 * layout as the library's public step type only because both describe the
 * same wiring-diagram step.
 *
 * Conventions (paper Sec. 2b): the state index has address bits
 * a(M)...a(2)a(1), a(1) the least significant.  Here bit b (0-based) of the
 * index is a(b+1); a step's 'goto' wire is target+1.  All state arithmetic
 * is FP64 complex; amplitudes are only moved, never combined, except in the
 * probability routine.  Compile with -ffp-contract=off.
 *
 * Every function names the passage it follows.  Readings of passages that
 * are garbled or silent are listed where they are used.
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double re, im;
} ocplx;

/* One wiring-diagram step: NOT on wire target+1 (Sec. 2e) when ctrl_mask
 * is 0, otherwise a NOT that fires when every control bit of the row index
 * equals the matching bit of ctrl_pol (Sec. 2b 'from' wire, Sec. 2g double
 * controls; more controls and negative polarity are this file's reading of
 * Sec. 2g, which leaves them open). */
typedef struct {
    uint32_t target;
    uint32_t reserved;
    uint64_t ctrl_mask;
    uint64_t ctrl_pol;
} ostep;

/* Error codes: 0 ok, -1 invalid argument. */
#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* A step is a wiring-diagram step on M wires only if its target wire
 * exists, is not also a control, and the polarity names only control
 * wires (Sec. 2a: one unit entry per row, symmetric matrix). */
static int step_ok(uint32_t M, const ostep *s)
{
    uint64_t all = (M >= 64) ? ~0ull : ((1ull << M) - 1ull);
    if (s->target >= M) return 0;
    if (s->reserved != 0) return 0;
    if (s->ctrl_mask & ~all) return 0;
    if ((s->ctrl_mask >> s->target) & 1ull) return 0;
    if (s->ctrl_pol & ~s->ctrl_mask) return 0;
    return 1;
}

int oracle_validate(uint32_t M, const ostep *steps, size_t L)
{
    if (M < 1 || M > 40) return ORACLE_EINVAL;
    for (size_t s = 0; s < L; ++s)
        if (!step_ok(M, &steps[s])) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* Does row i of the step's matrix sit in a toggled sub-matrix?  The
 * sub-matrix of size 2^goto containing row i is toggled when the control
 * wires read as the step demands (Sec. 2b, 2d, 2f, 2g). */
static int toggled(const ostep *s, uint64_t i)
{
    return (i & s->ctrl_mask) == s->ctrl_pol;
}

/*
 * Row array of one step, y(i) = column of the unit entry in row i
 * (Sec. 2b, 0-based rows here).  Built the paper's way: start from the
 * identity y(i) = i, then for every toggled 2^goto sub-matrix move the
 * rows of its upper half down by 2^(goto-1) and the rows of its lower half
 * up by 2^(goto-1) (the +/- 2^(goto-1) t(goto,i) updates of Sec. 2b-2d and
 * the closing formula of Sec. 2i).
 */
int oracle_step_row_array(uint32_t M, const ostep *s, int64_t *y)
{
    if (M > 30 || !step_ok(M, s)) return ORACLE_EINVAL;
    const int64_t n = (int64_t)1 << M;
    const int64_t half = (int64_t)1 << s->target; /* 2^(goto-1) */
    for (int64_t i = 0; i < n; ++i) y[i] = i;
    for (int64_t blk = 0; blk < n; blk += 2 * half) {
        for (int64_t r = 0; r < half; ++r) {
            int64_t upper = blk + r; /* row in the upper half */
            if (!toggled(s, (uint64_t)upper)) continue;
            y[upper] = y[upper] + half;
            y[upper + half] = y[upper + half] - half;
        }
    }
    return ORACLE_OK;
}

/*
 * Sparse permutation product exactly as Sec. 2h states it: with x the row
 * array of the product so far and y that of the next step, the new product
 * is x(i) <- y(x(i)); x starts as the identity (Summary of Method).
 * Steps are taken in the order given.  n_rows = 2^M entries in x.
 */
int oracle_paper_product(uint32_t M, const ostep *steps, size_t L, int64_t *x)
{
    if (M > 30 || oracle_validate(M, steps, L) != ORACLE_OK) return ORACLE_EINVAL;
    const int64_t n = (int64_t)1 << M;
    int64_t *y = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!y) return ORACLE_EINVAL;
    for (int64_t i = 0; i < n; ++i) x[i] = i;
    for (size_t s = 0; s < L; ++s) {
        oracle_step_row_array(M, &steps[s], y);
        for (int64_t i = 0; i < n; ++i) x[i] = y[x[i]];
    }
    free(y);
    return ORACLE_OK;
}

/*
 * Gather map of a wiring diagram: x such that k2(i) = k1(x(i)) gives
 * k2 = U_L ... U_1 k1 (steps[0] acts first, as in a physical circuit).
 *
 * Reading: the Sec. 2h rule x(i) <- y(x(i)) builds the product of the step
 * matrices in the order they are fed (product so far on the left), and
 * the final gather k2(i) = k1(x(i)) then applies that product.  Fed in
 * circuit order it yields U_1 U_2 ... U_L, the inverse of the circuit when
 * the step sequence is not a palindrome (each U_s is its own inverse,
 * Sec. 2a).  The rule is therefore fed the steps last-to-first.
 */
int oracle_gather_map(uint32_t M, const ostep *steps, size_t L, int64_t *x)
{
    if (M > 30 || oracle_validate(M, steps, L) != ORACLE_OK) return ORACLE_EINVAL;
    ostep *rev = (ostep *)malloc(sizeof(ostep) * (L ? L : 1));
    if (!rev) return ORACLE_EINVAL;
    for (size_t s = 0; s < L; ++s) rev[s] = steps[L - 1 - s];
    int rc = oracle_paper_product(M, rev, L, x);
    free(rev);
    return rc;
}

/* Output state from the product: k2(i) = k1(x(i)) for all i
 * (Sec. 2b closing formula; Summary of Method, last item). */
int oracle_gather(uint32_t M, const ocplx *k1, const int64_t *x, ocplx *k2)
{
    if (M > 30) return ORACLE_EINVAL;
    const int64_t n = (int64_t)1 << M;
    for (int64_t i = 0; i < n; ++i) k2[i] = k1[x[i]];
    return ORACLE_OK;
}

/*
 * Plain definition, one step at a time: k <- U_s k for s = steps[0], ...,
 * steps[L-1], where U_s is the symmetric permutation matrix of the step
 * (Sec. 2a).  U_s exchanges the two halves of every toggled 2^goto
 * sub-matrix (Sec. 2d), so applying it exchanges amplitude i with
 * amplitude i + 2^(goto-1) for every upper-half row i that is toggled.
 * In place; state length 2^M.
 */
int oracle_apply_circuit(uint32_t M, ocplx *k, const ostep *steps, size_t L)
{
    if (oracle_validate(M, steps, L) != ORACLE_OK || M > 36) return ORACLE_EINVAL;
    const uint64_t n = 1ull << M;
    for (size_t s = 0; s < L; ++s) {
        const ostep *st = &steps[s];
        const uint64_t half = 1ull << st->target;
        for (uint64_t i = 0; i < n; ++i) {
            if (i & half) continue; /* visit upper-half rows only */
            if (!toggled(st, i)) continue;
            ocplx tmp = k[i];
            k[i] = k[i + half];
            k[i + half] = tmp;
        }
    }
    return ORACLE_OK;
}

/*
 * One row of the gather map without materialising any array: x(i) for a
 * single output row i, following the same reading as oracle_gather_map
 * (the paper's row rule applied with the last step first).  Each step's
 * row map is evaluated by its +/- 2^(goto-1) form (Sec. 2i closing
 * formula): a toggled upper-half row moves down by 2^(goto-1), a toggled
 * lower-half row moves up.  This is what lets the oracle check single
 * outputs of states far too large to hold on the host.
 */
int oracle_source_rows(uint32_t M, const ostep *steps, size_t L,
                       const uint64_t *rows, size_t n_rows, uint64_t *src)
{
    if (oracle_validate(M, steps, L) != ORACLE_OK) return ORACLE_EINVAL;
    const uint64_t n = (M >= 64) ? ~0ull : (1ull << M);
    for (size_t r = 0; r < n_rows; ++r) {
        uint64_t i = rows[r];
        if (i >= n) return ORACLE_EINVAL;
        for (size_t s = L; s-- > 0;) {
            const ostep *st = &steps[s];
            if (!toggled(st, i)) continue;
            const uint64_t half = 1ull << st->target;
            if (i & half)
                i -= half; /* lower half of the sub-matrix */
            else
                i += half; /* upper half */
        }
        src[r] = i;
    }
    return ORACLE_OK;
}

/*
 * Input state generated from M qubits (App. 1): k1 is the Kronecker product
 * q_M (x) ... (x) q_2 (x) q_1, so k1(i) is the product of the component of
 * each qubit picked by the matching bit of i -- e.g. k1(5) = q3(1) q2(0) q1(1).
 * The factors are multiplied in that printed order, most significant qubit
 * first; each complex product is (ac - bd) + (ad + bc)i with every real
 * product and sum rounded separately.  q[2*b + v] is qubit b+1's component v.
 */
int oracle_product_state(uint32_t M, const ocplx *q, ocplx *k)
{
    if (M < 1 || M > 30) return ORACLE_EINVAL;
    const uint64_t n = 1ull << M;
    for (uint64_t i = 0; i < n; ++i) {
        ocplx acc = q[2 * (M - 1) + ((i >> (M - 1)) & 1u)];
        for (int b = (int)M - 2; b >= 0; --b) {
            const ocplx f = q[2 * b + ((i >> b) & 1u)];
            const double re = acc.re * f.re - acc.im * f.im;
            const double im = acc.re * f.im + acc.im * f.re;
            acc.re = re;
            acc.im = im;
        }
        k[i] = acc;
    }
    return ORACLE_OK;
}

/*
 * Basis-state probabilities |k(i)|^2 = re^2 + im^2 in FP64 (the state's
 * post-processing, Sec. 2b; amplitudes of arbitrary magnitude and phase,
 * Sec. 1).  Two products and one sum, no fused multiply-add.
 */
void oracle_probabilities(const ocplx *k, size_t n, double *p)
{
    for (size_t i = 0; i < n; ++i) {
        double a = k[i].re * k[i].re;
        double b = k[i].im * k[i].im;
        p[i] = a + b;
    }
}

/* Pairwise (cascade) summation of n doubles, the textbook method with error
 * growth O(log n); blocks of 64 are summed left to right. */
static double pairwise(const double *v, size_t n)
{
    if (n <= 64) {
        double s = 0.0;
        for (size_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    size_t h = n / 2;
    return pairwise(v, h) + pairwise(v + h, n - h);
}

double oracle_sum(const double *v, size_t n) { return pairwise(v, n); }
