/*
 * Plain C schoolbook oracle for c = a*b in Z_q[x]/(x^n+1), and in the cyclic
 * ring Z_q[x]/(x^n-1) (Sec. 2.1 names it as the other common ring): there
 * x^n = 1, so the products with i + k = j + n are added instead of
 * subtracted.
 *
 * TEST INFRASTRUCTURE ONLY: called by the test-suite, smoke() and the
 * cpu_baseline leg of bench.py through ctypes.  It shares nothing with the
 * CUDA library.
 *
 * It writes out the definition the paper gives (Sec. 2.1 (i) and the Sec. 2.2
 * fold rule): the coefficient of x^j is the sum of a_i*b_k over i+k = j minus
 * the sum of a_i*b_k over i+k = j+n, reduced once into [0, q).  Every product
 * a_i*b_k < 2^128 is formed exactly in unsigned __int128 and added to a
 * 192-bit accumulator (three 64-bit words), so nothing can overflow for any
 * n <= 2^62 and q < 2^64.  No blocking, no lazy reduction, no reordering.
 */
#include <stdint.h>
#include <stddef.h>

typedef unsigned __int128 u128;

typedef struct {
    uint64_t w0, w1, w2; /* value = w2*2^128 + w1*2^64 + w0 */
} acc192;

static void acc_add(acc192 *s, u128 p)
{
    uint64_t lo = (uint64_t)p;
    uint64_t hi = (uint64_t)(p >> 64);
    uint64_t t = s->w0 + lo;
    uint64_t c = t < lo;
    s->w0 = t;
    uint64_t u = s->w1 + hi;
    uint64_t c2 = u < hi;
    uint64_t v = u + c;
    c2 += v < u;
    s->w1 = v;
    s->w2 += c2;
}

/* value mod q by Horner's rule in base 2^64 */
static uint64_t acc_mod(const acc192 *s, uint64_t q)
{
    u128 r = s->w2 % q;
    r = ((r << 64) | s->w1) % q;
    r = ((r << 64) | s->w0) % q;
    return (uint64_t)r;
}

/* Coefficient j of one product: the low sum (i + k = j) and the wrapped
 * sum (i + k = j + n), combined with the wrap sign of the ring. */
static uint64_t coeff(const uint64_t *a, const uint64_t *b, uint64_t n, uint64_t q,
                      uint64_t j, int cyclic)
{
    acc192 low = {0, 0, 0}, wrap = {0, 0, 0};
    /* i + k = j : k = j - i for i <= j */
    for (uint64_t i = 0; i <= j; ++i)
        acc_add(&low, (u128)a[i] * b[j - i]);
    /* i + k = j + n : k = j + n - i for i > j */
    for (uint64_t i = j + 1; i < n; ++i)
        acc_add(&wrap, (u128)a[i] * b[j + n - i]);
    uint64_t p = acc_mod(&low, q), m = acc_mod(&wrap, q);
    if (cyclic)
        return (uint64_t)(((u128)p + m) % q);
    return p >= m ? p - m : (uint64_t)(((u128)p + q) - m);
}

/* One product: a, b, c are n-entry arrays of canonical residues. */
void oracle_negacyclic(const uint64_t *a, const uint64_t *b, uint64_t *c,
                       uint64_t n, uint64_t q)
{
    for (uint64_t j = 0; j < n; ++j)
        c[j] = coeff(a, b, n, q, j, 0);
}

void oracle_cyclic(const uint64_t *a, const uint64_t *b, uint64_t *c,
                   uint64_t n, uint64_t q)
{
    for (uint64_t j = 0; j < n; ++j)
        c[j] = coeff(a, b, n, q, j, 1);
}

/*
 * Batch over a [batch][k][n] layout (uint64 entries): products
 * first .. first+count-1, every prime of each.
 */
static void batch(const uint64_t *a, const uint64_t *b, uint64_t *c, uint64_t n,
                  const uint64_t *q_list, uint64_t k, uint64_t first, uint64_t count, int cyclic)
{
    for (uint64_t p = first; p < first + count; ++p)
        for (uint64_t j = 0; j < k; ++j) {
            size_t off = (size_t)((p * k + j) * n);
            for (uint64_t t = 0; t < n; ++t)
                c[off + t] = coeff(a + off, b + off, n, q_list[j], t, cyclic);
        }
}

void oracle_negacyclic_batch(const uint64_t *a, const uint64_t *b, uint64_t *c,
                             uint64_t n, const uint64_t *q_list, uint64_t k,
                             uint64_t first, uint64_t count)
{
    batch(a, b, c, n, q_list, k, first, count, 0);
}

void oracle_cyclic_batch(const uint64_t *a, const uint64_t *b, uint64_t *c,
                         uint64_t n, const uint64_t *q_list, uint64_t k,
                         uint64_t first, uint64_t count)
{
    batch(a, b, c, n, q_list, k, first, count, 1);
}

/* Only the listed output coefficients of one product (sampled parity). */
void oracle_negacyclic_coeffs(const uint64_t *a, const uint64_t *b, uint64_t n, uint64_t q,
                              const uint64_t *js, uint64_t count, uint64_t *out)
{
    for (uint64_t t = 0; t < count; ++t)
        out[t] = coeff(a, b, n, q, js[t], 0);
}

void oracle_cyclic_coeffs(const uint64_t *a, const uint64_t *b, uint64_t n, uint64_t q,
                          const uint64_t *js, uint64_t count, uint64_t *out)
{
    for (uint64_t t = 0; t < count; ++t)
        out[t] = coeff(a, b, n, q, js[t], 1);
}
