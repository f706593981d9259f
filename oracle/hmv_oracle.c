/*
 * CPU oracle for the multiprecision structured matrix-vector product
 * (Beliakov, "On fast matrix-vector multiplication with a Hankel matrix in
 * multiprecision arithmetics", arXiv:1402.5287).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * it exists so that tests, the smoke check and the benchmark's CPU baseline
 * can check the CUDA library against the plain definitions.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes, straight from the definitions (0-based indices):
 *   Hankel    (Sec. 1, matrix A_H):  y_i = sum_j a_{i+j} x_j,          len(a) = 2n-1
 *   Toeplitz  (Sec. 1, matrix A_T):  y_i = sum_j a_{n-1-i+j} x_j,      len(a) = 2n-1
 *   Circulant (Sec. 1, matrix A_C):  y_i = sum_j c_{(i-j) mod n} x_j,  len(c) = n
 * using the schoolbook product of Sec. 1 (summation over j; the printed
 * formula sums over the row index by a typo), with every multiplication and
 * addition done exactly on unsigned 32-bit limbs.  Positive and negative
 * products are summed into two separate exact accumulators and subtracted
 * once at the end.
 *
 * Number format: value = (neg ? -1 : 1) * M * 2^(E - b), 0 <= M < 2^b,
 * M in ceil(b/32) little-endian 32-bit limbs.  The exact integer result of a
 * row is Z_i = sum_j (+-M_a)(+-M_x), at scale 2^(E_a + E_x - 2b).
 *
 * Rounding (the paper leaves it unstated; reading recorded with the other
 * readings of the paper): b magnitude bits, round half to even on |Z|, and
 * the output exponent E_y is the least integer for which every rounded
 * mantissa stays below 2^b.  E_y is chosen from the exact Z, never from a
 * rounded value.  An all-zero result has E_y = E_a + E_x.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OK = 0, E_ARG = 1, E_MEM = 2, E_OVERFLOW = 3 };
enum { HANKEL = 0, TOEPLITZ = 1, CIRCULANT = 2 };

/* index into a[] of matrix entry (i, j), from the three matrix forms */
static int64_t entry_index(int kind, int64_t n, int64_t i, int64_t j) {
    if (kind == HANKEL) return i + j;
    if (kind == TOEPLITZ) return n - 1 - i + j;
    return ((i - j) % n + n) % n; /* circulant */
}

typedef struct {
    int kind, n, L, zl, a_len;
    const uint32_t *a, *x;
    const uint8_t *a_neg, *x_neg;
    const int32_t *rows;
    int nrows;
    uint32_t *z;
    uint8_t *z_neg;
    int next;
    pthread_mutex_t mu;
    int status;
} job_t;

/* Add the exact product u*v (L limbs each) into column sums.
 * lo[k] collects the low halves of limb products of weight k,
 * hi[k] the high halves of limb products of weight k (they weigh k+1). */
static void mul_accumulate(const uint32_t *u, const uint32_t *v, int L,
                           uint64_t *lo, uint64_t *hi) {
    for (int p = 0; p < L; ++p) {
        uint64_t up = u[p];
        if (up == 0) continue;
        uint64_t *lp = lo + p, *hp = hi + p;
        for (int q = 0; q < L; ++q) {
            uint64_t t = up * (uint64_t)v[q];
            lp[q] += (uint32_t)t;
            hp[q] += t >> 32;
        }
    }
}

/* Turn column sums into 32-bit limbs: out[k] for k < W. Returns 0 if the
 * value does not fit in W limbs. */
static int columns_to_limbs(const uint64_t *lo, const uint64_t *hi, int ncol,
                            uint32_t *out, int W) {
    uint64_t carry = 0; /* carry < 2^33 since every column sum < 2^63 */
    for (int k = 0; k < W; ++k) {
        uint64_t c = carry;
        uint64_t add_lo = (k < ncol) ? lo[k] : 0;
        uint64_t add_hi = (k >= 1 && k - 1 < ncol) ? hi[k - 1] : 0;
        /* sum the three parts in two halves to avoid any 64-bit overflow */
        uint64_t s_low = (c & 0xFFFFFFFFu) + (add_lo & 0xFFFFFFFFu) + (add_hi & 0xFFFFFFFFu);
        uint64_t s_high = (c >> 32) + (add_lo >> 32) + (add_hi >> 32) + (s_low >> 32);
        out[k] = (uint32_t)s_low;
        carry = s_high;
    }
    return carry == 0;
}

/* a - b for W-limb magnitudes, a >= b */
static void sub_limbs(const uint32_t *a, const uint32_t *b, uint32_t *out, int W) {
    int64_t borrow = 0;
    for (int k = 0; k < W; ++k) {
        int64_t d = (int64_t)a[k] - (int64_t)b[k] - borrow;
        borrow = d < 0;
        out[k] = (uint32_t)(d + (borrow ? ((int64_t)1 << 32) : 0));
    }
}

static int cmp_limbs(const uint32_t *a, const uint32_t *b, int W) {
    for (int k = W - 1; k >= 0; --k) {
        if (a[k] != b[k]) return a[k] > b[k] ? 1 : -1;
    }
    return 0;
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    const int L = J->L;
    const int ncol = 2 * L;
    const int W = J->zl;
    uint64_t *acc = (uint64_t *)calloc((size_t)4 * ncol, sizeof(uint64_t));
    uint32_t *P = (uint32_t *)calloc((size_t)2 * W, sizeof(uint32_t));
    if (!acc || !P) {
        pthread_mutex_lock(&J->mu);
        J->status = E_MEM;
        pthread_mutex_unlock(&J->mu);
        free(acc);
        free(P);
        return NULL;
    }
    uint32_t *N = P + W;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int r = J->next++;
        int stop = (r >= J->nrows) || J->status != OK;
        pthread_mutex_unlock(&J->mu);
        if (stop) break;
        int64_t i = J->rows[r];
        memset(acc, 0, (size_t)4 * ncol * sizeof(uint64_t));
        uint64_t *plo = acc, *phi = acc + ncol, *nlo = acc + 2 * ncol, *nhi = acc + 3 * ncol;
        for (int64_t j = 0; j < J->n; ++j) {
            int64_t k = entry_index(J->kind, J->n, i, j);
            const uint32_t *u = J->a + (size_t)k * L;
            const uint32_t *v = J->x + (size_t)j * L;
            int negative = (J->a_neg[k] != 0) != (J->x_neg[j] != 0);
            if (negative)
                mul_accumulate(u, v, L, nlo, nhi);
            else
                mul_accumulate(u, v, L, plo, phi);
        }
        int fit = columns_to_limbs(plo, phi, ncol, P, W) & columns_to_limbs(nlo, nhi, ncol, N, W);
        if (!fit) {
            pthread_mutex_lock(&J->mu);
            J->status = E_OVERFLOW;
            pthread_mutex_unlock(&J->mu);
            break;
        }
        uint32_t *z = J->z + (size_t)r * W;
        int c = cmp_limbs(P, N, W);
        if (c >= 0) {
            sub_limbs(P, N, z, W);
            J->z_neg[r] = 0;
        } else {
            sub_limbs(N, P, z, W);
            J->z_neg[r] = 1;
        }
    }
    free(acc);
    free(P);
    return NULL;
}

/*
 * Exact rows Z_i (magnitude in zl limbs + sign) of the structured product,
 * for the rows listed in rows[0..nrows).  a_len must be 2n-1 (Hankel,
 * Toeplitz) or n (circulant).  nthreads <= 0 means 1.
 */
int oracle_exact_rows(int kind, int n, int b,
                      const uint32_t *a_limbs, const uint8_t *a_neg, int a_len,
                      const uint32_t *x_limbs, const uint8_t *x_neg,
                      int nrows, const int32_t *rows,
                      int zl, uint32_t *z_mag, uint8_t *z_neg, int nthreads) {
    if (n < 1 || b < 1 || kind < 0 || kind > 2 || nrows < 0) return E_ARG;
    int want_len = (kind == CIRCULANT) ? n : 2 * n - 1;
    if (a_len != want_len) return E_ARG;
    int L = (b + 31) / 32;
    if (zl < 2 * L + 1) return E_ARG;
    if ((int64_t)n * L >= ((int64_t)1 << 30)) return E_ARG; /* column sums must stay < 2^63 */
    for (int r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= n) return E_ARG;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nrows && nrows > 0) nthreads = nrows;
    job_t J;
    memset(&J, 0, sizeof J);
    J.kind = kind; J.n = n; J.L = L; J.zl = zl; J.a_len = a_len;
    J.a = a_limbs; J.x = x_limbs; J.a_neg = a_neg; J.x_neg = x_neg;
    J.rows = rows; J.nrows = nrows; J.z = z_mag; J.z_neg = z_neg;
    pthread_mutex_init(&J.mu, NULL);
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th) return E_MEM;
    int started = 0;
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[started], NULL, worker, &J) == 0) ++started;
    /* the calling thread works too */
    worker(&J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    return J.status;
}

/* number of significant bits of a W-limb magnitude (0 for zero) */
static int64_t bitlength(const uint32_t *m, int W) {
    for (int k = W - 1; k >= 0; --k) {
        if (m[k]) {
            int64_t bl = 32 * (int64_t)k;
            uint32_t v = m[k];
            while (v) { ++bl; v >>= 1; }
            return bl;
        }
    }
    return 0;
}

static int get_bit(const uint32_t *m, int W, int64_t pos) {
    if (pos < 0 || pos >= 32 * (int64_t)W) return 0;
    return (m[pos >> 5] >> (pos & 31)) & 1;
}

/* any bit set strictly below position pos */
static int any_below(const uint32_t *m, int W, int64_t pos) {
    for (int64_t k = 0; k < W && 32 * k < pos; ++k) {
        uint32_t v = m[k];
        int64_t top = pos - 32 * k; /* bits [0, top) of this limb count */
        if (top < 32) v &= (top <= 0) ? 0u : ((1u << top) - 1u);
        if (v) return 1;
    }
    return 0;
}

/* RNE(|z| / 2^t) into out (Lb limbs), t may be <= 0 (exact left shift).
 * Returns 1 if the rounded value reaches 2^b. */
static int round_one(const uint32_t *z, int W, int64_t t, int b, uint32_t *out, int Lb) {
    memset(out, 0, (size_t)Lb * sizeof(uint32_t));
    /* out bit p = z bit (p + t) for p < b */
    for (int64_t p = 0; p < b; ++p)
        if (get_bit(z, W, p + t)) out[p >> 5] |= 1u << (p & 31);
    /* bits of z at or above b + t must be zero (caller guarantees) */
    if (t > 0) {
        int half = get_bit(z, W, t - 1);
        int sticky = any_below(z, W, t - 1);
        int odd = out[0] & 1u;
        if (half && (sticky || odd)) {
            /* increment; out has room for 2^b */
            for (int k = 0; k < Lb; ++k) {
                out[k] += 1u;
                if (out[k] != 0) break;
            }
        }
    }
    return bitlength(out, Lb) > b;
}

/*
 * Round exact rows to b-bit mantissas with one shared exponent.
 * e_in = E_a + E_x.  Writes y_limbs (count x ceil(b/32)), y_neg, *e_out.
 */
int oracle_round(int count, int zl, const uint32_t *z_mag, const uint8_t *z_neg,
                 int b, int e_in, uint32_t *y_limbs, uint8_t *y_neg, int32_t *e_out) {
    if (count < 0 || zl < 1 || b < 1) return E_ARG;
    int Lb = (b + 31) / 32;
    /* Lb limbs hold 32*Lb >= b bits; a carry to 2^b needs bit b, which fits
     * unless b is a multiple of 32, so use a scratch of Lb + 1 limbs. */
    uint32_t *tmp = (uint32_t *)calloc((size_t)Lb + 1, sizeof(uint32_t));
    if (!tmp) return E_MEM;
    int64_t B = 0;
    for (int r = 0; r < count; ++r) {
        int64_t bl = bitlength(z_mag + (size_t)r * zl, zl);
        if (bl > B) B = bl;
    }
    if (B == 0) {
        memset(y_limbs, 0, (size_t)count * Lb * sizeof(uint32_t));
        memset(y_neg, 0, (size_t)count);
        *e_out = e_in;
        free(tmp);
        return OK;
    }
    int64_t t = B - b;
    for (int pass = 0; pass < 2; ++pass) {
        int overflow = 0;
        for (int r = 0; r < count && !overflow; ++r)
            overflow |= round_one(z_mag + (size_t)r * zl, zl, t, b, tmp, Lb + 1);
        if (!overflow) break;
        t += 1; /* only the largest rows can round up to 2^b: one step suffices */
    }
    for (int r = 0; r < count; ++r) {
        int ov = round_one(z_mag + (size_t)r * zl, zl, t, b, tmp, Lb + 1);
        if (ov) { free(tmp); return E_OVERFLOW; }
        memcpy(y_limbs + (size_t)r * Lb, tmp, (size_t)Lb * sizeof(uint32_t));
        int zero = bitlength(tmp, Lb) == 0;
        y_neg[r] = zero ? 0 : (z_neg[r] ? 1 : 0);
    }
    int64_t e = (int64_t)e_in + t - b;
    *e_out = (int32_t)e;
    free(tmp);
    return OK;
}

/* Round with a given shift t (used when only a sample of rows is known and
 * the exponent comes from elsewhere). Returns E_OVERFLOW if a row reaches 2^b. */
int oracle_round_fixed_shift(int count, int zl, const uint32_t *z_mag, const uint8_t *z_neg,
                             int b, int64_t t, uint32_t *y_limbs, uint8_t *y_neg) {
    if (count < 0 || zl < 1 || b < 1) return E_ARG;
    int Lb = (b + 31) / 32;
    uint32_t *tmp = (uint32_t *)calloc((size_t)Lb + 1, sizeof(uint32_t));
    if (!tmp) return E_MEM;
    for (int r = 0; r < count; ++r) {
        const uint32_t *z = z_mag + (size_t)r * zl;
        if (bitlength(z, zl) > (int64_t)b + t) { free(tmp); return E_OVERFLOW; }
        int ov = round_one(z, zl, t, b, tmp, Lb + 1);
        if (ov) { free(tmp); return E_OVERFLOW; }
        memcpy(y_limbs + (size_t)r * Lb, tmp, (size_t)Lb * sizeof(uint32_t));
        y_neg[r] = bitlength(tmp, Lb) == 0 ? 0 : (z_neg[r] ? 1 : 0);
    }
    free(tmp);
    return OK;
}
