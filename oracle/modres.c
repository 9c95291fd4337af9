/* O2: an independent modular resultant over Z on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU legs of
 * bench.py load this file's library; the resultant library never does, and
 * this file shares no code, header, table or constant with it.
 *
 * What it computes (paper, Section 3.1): R(x) = res(f, g, y) in Z[x], the
 * determinant of the (m_y + n_y)-square Sylvester matrix whose first n_y rows
 * hold the y-coefficients f_{m_y}, ..., f_0 of f (each row shifted one column
 * right of the previous) and whose last m_y rows hold g_{n_y}, ..., g_0 the
 * same way; m_y, n_y are the y-degrees of f and g over Z[x].
 *
 * How (the modular method of Section 4.1, in its plainest form):
 *   1. a degree bound D for R and a coefficient bound 2^B (Section 3.1 and the
 *      Hadamard inequality, see o2_plan_pair);
 *   2. K primes of this file's own table (the largest primes below
 *      2^31 - 2^20, descending) with prod p > 2^(B+1);
 *   3. per prime p and per point x = 0, 1, ..., D: the entries f_j(x), g_j(x)
 *      mod p (Horner), then det S(x) mod p -- by the textbook Euclidean
 *      algorithm when both leading coefficients survive at x (then the
 *      formal degrees are the actual ones and the Sylvester determinant is
 *      the resultant of the two univariate polynomials), otherwise by
 *      Gaussian elimination of the formal Sylvester matrix itself;
 *   4. R mod p by Lagrange interpolation through the D + 1 values;
 *   5. R by the constructive Chinese remainder theorem on a small bignum, in
 *      the symmetric range (-P/2, P/2].
 * Arithmetic is 64-bit products reduced with the C remainder operator; no
 * Montgomery or Barrett form, no blocking, no fusion.
 *
 * Input layout: f_ij in two's complement 32-bit limbs, little-endian,
 * coeffs[((i * (deg_y + 1)) + j) * limbs + l], i the power of x.
 *
 * O2_PLANT (undefined in every normal build): the CPU tests compile this
 * file a second time with O2_PLANT = 1..7 to plant one plausible mistake
 * each -- a dropped Euclid sign, a wrong leading-coefficient power, a dropped
 * Lagrange sign, no symmetric range, g-rows first, a degree bound one too
 * small, a sign-blind coefficient reduction -- and check that the pins
 * catch every one.
 */
#ifndef O2_PLANT
#define O2_PLANT 0
#endif
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O2_OK 0
#define O2_ERR_ARG (-1)
#define O2_ERR_NOMEM (-2)
#define O2_ERR_BOUND (-3) /* a CRT value outside the coefficient bound */
#define O2_ERR_PRIMES (-4)

#define O2_PRIME_TOP ((1u << 31) - (1u << 20)) /* every table prime is below this */
#define O2_MAX_PRIMES 8192

typedef struct {
    int32_t deg_x, deg_y, limbs;
    const uint32_t *coeffs;
} o2_poly;

typedef struct {
    int32_t m_y, n_y;  /* y-degrees after trimming (-1: the zero polynomial) */
    int32_t m_x, n_x;  /* x-degrees after trimming */
    int32_t D;         /* deg R <= D; D + 1 evaluation points */
    int32_t bits;      /* B: every |coefficient of R| <= 2^B */
    int32_t nprimes;   /* K */
    int32_t out_limbs; /* 32-bit limbs per output coefficient */
    int32_t zero;      /* 1: f or g is zero, so R = 0 without any work */
    int32_t pad;
} o2_plan;

/* ------------------------------------------------------------ Z_p helpers */

static inline uint32_t mulm(uint32_t a, uint32_t b, uint32_t p) { return (uint32_t)((uint64_t)a * b % p); }
static inline uint32_t addm(uint32_t a, uint32_t b, uint32_t p) {
    uint32_t s = a + b; /* a, b < p < 2^31 */
    return s >= p ? s - p : s;
}
static inline uint32_t subm(uint32_t a, uint32_t b, uint32_t p) { return a >= b ? a - b : a + (p - b); }
static inline uint32_t negm(uint32_t a, uint32_t p) { return a ? p - a : 0; }

/* a^-1 mod p by the extended Euclidean algorithm (a != 0 mod p). */
static uint32_t invm(uint32_t a, uint32_t p) {
    int64_t r0 = p, r1 = a % p, s0 = 0, s1 = 1;
    while (r1) {
        int64_t q = r0 / r1, t;
        t = r0 - q * r1; r0 = r1; r1 = t;
        t = s0 - q * s1; s0 = s1; s1 = t;
    }
    /* r0 = gcd = 1; s0 * a = 1 mod p */
    s0 %= (int64_t)p;
    if (s0 < 0) s0 += p;
    return (uint32_t)s0;
}

static uint32_t powm(uint32_t a, int64_t e, uint32_t p) {
    uint32_t r = 1 % p;
    while (e > 0) {
        if (e & 1) r = mulm(r, a, p);
        a = mulm(a, a, p);
        e >>= 1;
    }
    return r;
}

/* --------------------------------------------------------------- primes */

static uint32_t g_primes[O2_MAX_PRIMES];
static int g_nprimes = 0;
static pthread_once_t g_primes_once = PTHREAD_ONCE_INIT;

/* The table: the O2_MAX_PRIMES largest primes below 2^31 - 2^20, in
 * descending order, each tested by trial division by every prime up to
 * sqrt(2^31) (46341). */
static void primes_init(void) {
    enum { LIM = 46341 };
    static unsigned char comp[LIM + 1];
    static uint32_t small[LIM];
    int ns = 0;
    for (uint32_t i = 2; i <= LIM; i++) {
        if (comp[i]) continue;
        small[ns++] = i;
        for (uint32_t j = i * i; j <= LIM; j += i) comp[j] = 1;
    }
    uint32_t c = O2_PRIME_TOP - 1; /* odd: 2^31 - 2^20 - 1 */
    while (g_nprimes < O2_MAX_PRIMES) {
        int is_p = 1;
        for (int k = 0; k < ns && (uint64_t)small[k] * small[k] <= c; k++)
            if (c % small[k] == 0) { is_p = 0; break; }
        if (is_p) g_primes[g_nprimes++] = c;
        c -= 2;
    }
}

uint32_t o2_prime(int32_t k) {
    pthread_once(&g_primes_once, primes_init);
    if (k < 0 || k >= g_nprimes) return 0;
    return g_primes[k];
}

/* ------------------------------------------------------------ input access */

static const uint32_t *coef_ptr(const o2_poly *f, int i, int j) {
    return f->coeffs + ((size_t)i * (f->deg_y + 1) + j) * f->limbs;
}

static int coef_is_zero(const o2_poly *f, int i, int j) {
    const uint32_t *c = coef_ptr(f, i, j);
    for (int l = 0; l < f->limbs; l++)
        if (c[l]) return 0;
    return 1;
}

/* |v| of a two's-complement limb vector, as L unsigned limbs (L = limbs). */
static int abs_limbs(const uint32_t *c, int L, uint32_t *mag) {
    int neg = (c[L - 1] >> 31) & 1;
    uint64_t carry = 1;
    for (int l = 0; l < L; l++) {
        if (neg) {
            uint64_t s = (uint64_t)(uint32_t)~c[l] + carry;
            mag[l] = (uint32_t)s;
            carry = s >> 32;
        } else {
            mag[l] = c[l];
        }
    }
    return neg;
}

/* f_ij mod p: Horner over the magnitude's limbs from the top, then the sign. */
static uint32_t coef_mod(const o2_poly *f, int i, int j, uint32_t p, uint32_t *tmp) {
    int neg = abs_limbs(coef_ptr(f, i, j), f->limbs, tmp);
    uint64_t v = 0;
    for (int l = f->limbs - 1; l >= 0; l--) v = ((v << 32) | tmp[l]) % p;
    if (O2_PLANT == 7) neg = 0;
    return neg ? negm((uint32_t)v, p) : (uint32_t)v;
}

/* ------------------------------------------------------------ tiny bignum */
/* Non-negative integers as little-endian 32-bit limbs with an explicit
 * length (no leading zero limbs; length 0 is the number 0). */

static int bn_norm(const uint32_t *a, int n) {
    while (n > 0 && a[n - 1] == 0) n--;
    return n;
}

static uint32_t bn_mod_small(const uint32_t *a, int n, uint32_t p) {
    uint64_t v = 0;
    for (int l = n - 1; l >= 0; l--) v = ((v << 32) | a[l]) % p;
    return (uint32_t)v;
}

/* out[0..n] = a[0..n) * m; returns the new length */
static int bn_mul_small(const uint32_t *a, int n, uint32_t m, uint32_t *out) {
    uint64_t carry = 0;
    for (int l = 0; l < n; l++) {
        uint64_t t = (uint64_t)a[l] * m + carry;
        out[l] = (uint32_t)t;
        carry = t >> 32;
    }
    out[n] = (uint32_t)carry;
    return bn_norm(out, n + 1);
}

/* x += P * t, x has room for max(nx, nP + 1) + 1 limbs; returns new length */
static int bn_addmul(uint32_t *x, int nx, const uint32_t *P, int nP, uint32_t t) {
    int n = nx > nP + 1 ? nx : nP + 1;
    for (int l = nx; l <= n; l++) x[l] = 0;
    uint64_t carry = 0;
    for (int l = 0; l < nP; l++) {
        uint64_t s = (uint64_t)P[l] * t + x[l] + carry;
        x[l] = (uint32_t)s;
        carry = s >> 32;
    }
    for (int l = nP; l <= n && carry; l++) {
        uint64_t s = (uint64_t)x[l] + carry;
        x[l] = (uint32_t)s;
        carry = s >> 32;
    }
    return bn_norm(x, n + 1);
}

static int bn_cmp(const uint32_t *a, int na, const uint32_t *b, int nb) {
    if (na != nb) return na < nb ? -1 : 1;
    for (int l = na - 1; l >= 0; l--)
        if (a[l] != b[l]) return a[l] < b[l] ? -1 : 1;
    return 0;
}

/* out = a - b for a >= b; returns the length */
static int bn_sub(const uint32_t *a, int na, const uint32_t *b, int nb, uint32_t *out) {
    int64_t borrow = 0;
    for (int l = 0; l < na; l++) {
        int64_t s = (int64_t)a[l] - (l < nb ? b[l] : 0) - borrow;
        borrow = s < 0;
        out[l] = (uint32_t)(s + (borrow ? ((int64_t)1 << 32) : 0));
    }
    return bn_norm(out, na);
}

static int bn_bitlen(const uint32_t *a, int n) {
    if (n == 0) return 0;
    return 32 * (n - 1) + (32 - __builtin_clz(a[n - 1]));
}

/* out = a * b (schoolbook); out has na + nb limbs; returns the length */
static int bn_mul(const uint32_t *a, int na, const uint32_t *b, int nb, uint32_t *out) {
    memset(out, 0, sizeof(uint32_t) * (size_t)(na + nb));
    for (int i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < nb; j++) {
            uint64_t t = (uint64_t)a[i] * b[j] + out[i + j] + carry;
            out[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        out[i + nb] = (uint32_t)carry;
    }
    return bn_norm(out, na + nb);
}

/* out = a + b; out has max(na, nb) + 1 limbs; returns the length */
static int bn_add(const uint32_t *a, int na, const uint32_t *b, int nb, uint32_t *out) {
    int n = na > nb ? na : nb;
    uint64_t carry = 0;
    for (int l = 0; l < n; l++) {
        uint64_t s = (uint64_t)(l < na ? a[l] : 0) + (l < nb ? b[l] : 0) + carry;
        out[l] = (uint32_t)s;
        carry = s >> 32;
    }
    out[n] = (uint32_t)carry;
    return bn_norm(out, n + 1);
}

/* ------------------------------------------------------------------ plan */

static void degrees(const o2_poly *f, int *dx, int *dy, int *tdeg) {
    *dx = *dy = *tdeg = -1;
    for (int i = 0; i <= f->deg_x; i++)
        for (int j = 0; j <= f->deg_y; j++)
            if (!coef_is_zero(f, i, j)) {
                if (i > *dx) *dx = i;
                if (j > *dy) *dy = j;
                if (i + j > *tdeg) *tdeg = i + j;
            }
}

/* Bit length of S_f = sum_j ||f_j||_1^2 (f_j the y-coefficients of f, ||.||_1
 * the sum of absolute values of a Z[x] polynomial's coefficients), exactly.
 * Returns -1 on allocation failure. */
static int row_norm_bits(const o2_poly *f, int dx, int dy) {
    int L = f->limbs;
    int nl1 = L + 2, nsq = 2 * nl1 + 1;
    uint32_t *mag = malloc(sizeof(uint32_t) * (size_t)L);
    uint32_t *l1 = calloc((size_t)nl1 + 1, sizeof(uint32_t));
    uint32_t *t = calloc((size_t)nl1 + 1, sizeof(uint32_t));
    uint32_t *sq = calloc((size_t)nsq + 1, sizeof(uint32_t));
    uint32_t *S = calloc((size_t)nsq + 2, sizeof(uint32_t));
    uint32_t *S2 = calloc((size_t)nsq + 2, sizeof(uint32_t));
    int bits = -1;
    if (!mag || !l1 || !t || !sq || !S || !S2) goto done;
    int nS = 0;
    for (int j = 0; j <= dy; j++) {
        int n1 = 0;
        for (int i = 0; i <= dx; i++) {
            abs_limbs(coef_ptr(f, i, j), L, mag);
            int nm = bn_norm(mag, L);
            n1 = bn_add(l1, n1, mag, nm, t);
            memcpy(l1, t, sizeof(uint32_t) * (size_t)(n1 ? n1 : 1));
        }
        int ns = bn_mul(l1, n1, l1, n1, sq);
        nS = bn_add(S, nS, sq, ns, S2);
        memcpy(S, S2, sizeof(uint32_t) * (size_t)(nS ? nS : 1));
        memset(l1, 0, sizeof(uint32_t) * ((size_t)nl1 + 1));
    }
    bits = bn_bitlen(S, nS);
done:
    free(mag); free(l1); free(t); free(sq); free(S); free(S2);
    return bits;
}

/* Plan of one pair.
 *  - degrees: m_y, n_y, m_x, n_x of the nonzero coefficients; f or g zero
 *    gives R = 0 (the paper assumes both nonzero).
 *  - D = min(m_x n_y + n_x m_y, tdeg f * tdeg g): every term of the Leibniz
 *    expansion of S multiplies n_y entries of x-degree <= m_x and m_y
 *    entries of x-degree <= n_x; Section 3.1 gives the second form.
 *  - B: on |x| = 1 an f-row of S(x) has squared length
 *    sum_j |f_j(x)|^2 <= S_f, so Hadamard's inequality gives
 *    |R(x)| <= S_f^(n_y/2) S_g^(m_y/2) < 2^((n_y bits(S_f) + m_y bits(S_g))/2),
 *    and each coefficient of R, a Fourier coefficient of R on the unit
 *    circle, is at most max |R(x)| there.  B is that exponent rounded up.
 *  - K primes, each above 2^30, so prod p > 2^(30 K) >= 2^(B+2).
 *  - out_limbs holds any value of the symmetric range of prod p < 2^(31 K). */
int o2_plan_pair(const o2_poly *f, const o2_poly *g, o2_plan *pl) {
    if (!f || !g || !pl || f->limbs < 1 || g->limbs < 1 || f->deg_x < 0 || f->deg_y < 0 ||
        g->deg_x < 0 || g->deg_y < 0 || !f->coeffs || !g->coeffs)
        return O2_ERR_ARG;
    memset(pl, 0, sizeof(*pl));
    int tf, tg;
    degrees(f, &pl->m_x, &pl->m_y, &tf);
    degrees(g, &pl->n_x, &pl->n_y, &tg);
    if (pl->m_y < 0 || pl->n_y < 0) {
        pl->zero = 1;
        pl->D = -1;
        pl->out_limbs = 1;
        return O2_OK;
    }
    int64_t d1 = (int64_t)pl->m_x * pl->n_y + (int64_t)pl->n_x * pl->m_y;
    int64_t d2 = (int64_t)tf * tg;
    pl->D = (int32_t)(d1 < d2 ? d1 : d2);
    if (O2_PLANT == 6 && pl->D > 0) pl->D -= 1;
    int bf = row_norm_bits(f, pl->m_x, pl->m_y), bg = row_norm_bits(g, pl->n_x, pl->n_y);
    if (bf < 0 || bg < 0) return O2_ERR_NOMEM;
    int64_t twoB = (int64_t)pl->n_y * bf + (int64_t)pl->m_y * bg;
    pl->bits = (int32_t)((twoB + 1) / 2);
    pl->nprimes = (pl->bits + 1) / 30 + 1;
    if (pl->nprimes > O2_MAX_PRIMES) return O2_ERR_PRIMES;
    pl->out_limbs = (31 * pl->nprimes + 31) / 32;
    return O2_OK;
}

/* -------------------------------------------------- one image, two ways */

/* res(A, B) mod p for A of degree a, B of degree b with nonzero leading
 * coefficients, by the Euclidean algorithm and the textbook identities
 *   res(A, B) = (-1)^(a b) res(B, A),
 *   res(A, B) = (-1)^(a b) lc(B)^(a - r) res(B, A mod B)   (a >= b > 0, r = deg(A mod B)),
 *   res(A, B) = 0 if A mod B = 0 and b > 0,   res(A, c) = c^a for a constant c.
 * A and B are overwritten. */
static uint32_t res_euclid(uint32_t *A, int a, uint32_t *B, int b, uint32_t p) {
    uint32_t acc = 1;
    for (;;) {
        if (a < b) {
            uint32_t *t = A; A = B; B = t;
            int d = a; a = b; b = d;
            if ((a & 1) && (b & 1)) acc = negm(acc, p);
        }
        if (b == 0) return mulm(acc, powm(B[0], a, p), p);
        uint32_t inv = invm(B[b], p);
        for (int k = a; k >= b; k--) {
            uint32_t q = mulm(A[k], inv, p);
            if (q)
                for (int i = 0; i <= b; i++) A[k - b + i] = subm(A[k - b + i], mulm(q, B[i], p), p);
        }
        int r = b - 1;
        while (r >= 0 && A[r] == 0) r--;
        if (r < 0) return 0;
        if ((a & 1) && (b & 1) && O2_PLANT != 1) acc = negm(acc, p);
        acc = mulm(acc, powm(B[b], a - r - (O2_PLANT == 2), p), p);
        uint32_t *t = A; A = B; B = t; /* (A, B) <- (B, A mod B) */
        a = b;
        b = r;
    }
}

/* det of an n x n matrix over Z_p by Gaussian elimination with row swaps;
 * M is overwritten. */
static uint32_t det_gauss(uint32_t *M, int n, uint32_t p) {
    uint32_t det = 1;
    for (int k = 0; k < n; k++) {
        int piv = -1;
        for (int i = k; i < n; i++)
            if (M[(size_t)i * n + k]) { piv = i; break; }
        if (piv < 0) return 0;
        if (piv != k) {
            for (int j = 0; j < n; j++) {
                uint32_t t = M[(size_t)k * n + j];
                M[(size_t)k * n + j] = M[(size_t)piv * n + j];
                M[(size_t)piv * n + j] = t;
            }
            det = negm(det, p);
        }
        uint32_t pk = M[(size_t)k * n + k];
        det = mulm(det, pk, p);
        uint32_t inv = invm(pk, p);
        for (int i = k + 1; i < n; i++) {
            uint32_t fct = mulm(M[(size_t)i * n + k], inv, p);
            if (!fct) continue;
            for (int j = k; j < n; j++)
                M[(size_t)i * n + j] = subm(M[(size_t)i * n + j], mulm(fct, M[(size_t)k * n + j], p), p);
        }
    }
    return det;
}

/* The formal Sylvester matrix of Section 3.1 with entries F_j = f_j(x) mod p
 * (j = 0..my) and G_j, then its determinant. */
static uint32_t res_sylvester(const uint32_t *F, int my, const uint32_t *G, int ny, uint32_t p, uint32_t *M) {
    int r = my + ny;
    if (r == 0) return 1 % p;
    memset(M, 0, sizeof(uint32_t) * (size_t)r * r);
    int f0 = O2_PLANT == 5 ? my : 0, g0 = O2_PLANT == 5 ? 0 : ny; /* first f-row, first g-row */
    for (int row = 0; row < ny; row++)
        for (int k = 0; k <= my; k++) M[(size_t)(f0 + row) * r + row + k] = F[my - k];
    for (int row = 0; row < my; row++)
        for (int k = 0; k <= ny; k++) M[(size_t)(g0 + row) * r + row + k] = G[ny - k];
    return det_gauss(M, r, p);
}

/* --------------------------------------------------- interpolation mod p */

/* The polynomial c of degree < N with c(i) = z[i] for the points
 * i = 0, 1, ..., N - 1 (N < p), by Lagrange's formula
 *   c(x) = sum_i z_i / prod_{j != i} (i - j) * M(x) / (x - i),   M(x) = prod_j (x - j),
 * where prod_{j != i} (i - j) = i! (N - 1 - i)! (-1)^(N - 1 - i), and each
 * M(x) / (x - i) comes from synthetic division.  Scratch: M (N + 1 words),
 * fact and ifact (N words each). */
static void lagrange(const uint32_t *z, int N, uint32_t p, uint32_t *c, uint32_t *M, uint32_t *fact,
                     uint32_t *ifact) {
    memset(M, 0, sizeof(uint32_t) * (size_t)(N + 1));
    M[0] = 1 % p;
    for (int i = 0; i < N; i++) { /* M <- M * (x - i), degree i -> i + 1 */
        uint32_t xi = (uint32_t)i % p;
        for (int k = i + 1; k >= 1; k--) M[k] = subm(M[k - 1], mulm(xi, M[k], p), p);
        M[0] = negm(mulm(xi, M[0], p), p);
    }
    fact[0] = 1 % p;
    for (int i = 1; i < N; i++) fact[i] = mulm(fact[i - 1], (uint32_t)i, p);
    ifact[N - 1] = invm(fact[N - 1], p);
    for (int i = N - 1; i >= 1; i--) ifact[i - 1] = mulm(ifact[i], (uint32_t)i, p);
    memset(c, 0, sizeof(uint32_t) * (size_t)N);
    for (int i = 0; i < N; i++) {
        uint32_t w = mulm(z[i], mulm(ifact[i], ifact[N - 1 - i], p), p);
        if (((N - 1 - i) & 1) && O2_PLANT != 3) w = negm(w, p);
        if (!w) continue;
        uint32_t xi = (uint32_t)i, q = M[N]; /* quotient of M by (x - i), top down */
        c[N - 1] = addm(c[N - 1], mulm(w, q, p), p);
        for (int k = N - 1; k >= 1; k--) {
            q = addm(M[k], mulm(xi, q, p), p);
            c[k - 1] = addm(c[k - 1], mulm(w, q, p), p);
        }
    }
}

/* ------------------------------------------------- one (pair, prime) task */

typedef struct {
    uint32_t *fr, *gr, *F, *G, *A, *B, *M, *fact, *ifact, *z, *tmp;
    uint32_t *syl;
    size_t syl_words;
} scratch;

static void scratch_free(scratch *s) {
    free(s->fr); free(s->gr); free(s->F); free(s->G); free(s->A); free(s->B); free(s->M);
    free(s->fact); free(s->ifact); free(s->z); free(s->tmp); free(s->syl);
    memset(s, 0, sizeof(*s));
}

static int scratch_alloc(scratch *s, const o2_poly *f, const o2_poly *g, const o2_plan *pl) {
    memset(s, 0, sizeof(*s));
    int N = pl->D + 1, w = (pl->m_y > pl->n_y ? pl->m_y : pl->n_y) + 1;
    int L = f->limbs > g->limbs ? f->limbs : g->limbs;
    s->fr = malloc(sizeof(uint32_t) * (size_t)(pl->m_x + 1) * (pl->m_y + 1));
    s->gr = malloc(sizeof(uint32_t) * (size_t)(pl->n_x + 1) * (pl->n_y + 1));
    s->F = malloc(sizeof(uint32_t) * (size_t)w);
    s->G = malloc(sizeof(uint32_t) * (size_t)w);
    s->A = malloc(sizeof(uint32_t) * (size_t)w);
    s->B = malloc(sizeof(uint32_t) * (size_t)w);
    s->M = malloc(sizeof(uint32_t) * (size_t)(N + 1));
    s->fact = malloc(sizeof(uint32_t) * (size_t)N);
    s->ifact = malloc(sizeof(uint32_t) * (size_t)N);
    s->z = malloc(sizeof(uint32_t) * (size_t)N);
    s->tmp = malloc(sizeof(uint32_t) * (size_t)L);
    if (!s->fr || !s->gr || !s->F || !s->G || !s->A || !s->B || !s->M || !s->fact || !s->ifact || !s->z ||
        !s->tmp) {
        scratch_free(s);
        return O2_ERR_NOMEM;
    }
    return O2_OK;
}

/* f_ij mod p into fr[j * (m_x + 1) + i] (one row per power of y). */
static void reduce_poly(const o2_poly *f, int dx, int dy, uint32_t p, uint32_t *fr, uint32_t *tmp) {
    for (int j = 0; j <= dy; j++)
        for (int i = 0; i <= dx; i++) fr[(size_t)j * (dx + 1) + i] = coef_mod(f, i, j, p, tmp);
}

/* F_j = f_j(x) mod p for j = 0..dy, Horner in x. */
static void eval_rows(const uint32_t *fr, int dx, int dy, uint32_t x, uint32_t p, uint32_t *F) {
    for (int j = 0; j <= dy; j++) {
        const uint32_t *row = fr + (size_t)j * (dx + 1);
        uint32_t v = 0;
        for (int i = dx; i >= 0; i--) v = addm(mulm(v, x, p), row[i], p);
        F[j] = v;
    }
}

/* det S(x) mod p for one point, given the reduced coefficients. */
static int image_at(scratch *s, const o2_plan *pl, uint32_t p, uint32_t x, uint32_t *out) {
    int my = pl->m_y, ny = pl->n_y;
    eval_rows(s->fr, pl->m_x, my, x, p, s->F);
    eval_rows(s->gr, pl->n_x, ny, x, p, s->G);
    if (s->F[my] && s->G[ny]) {
        memcpy(s->A, s->F, sizeof(uint32_t) * (size_t)(my + 1));
        memcpy(s->B, s->G, sizeof(uint32_t) * (size_t)(ny + 1));
        *out = res_euclid(s->A, my, s->B, ny, p);
        return O2_OK;
    }
    size_t r = (size_t)(my + ny);
    if (r * r > s->syl_words) {
        free(s->syl);
        s->syl = malloc(sizeof(uint32_t) * (r ? r * r : 1));
        if (!s->syl) return O2_ERR_NOMEM;
        s->syl_words = r * r;
    }
    *out = res_sylvester(s->F, my, s->G, ny, p, s->syl);
    return O2_OK;
}

/* R mod p: the D + 1 images at x = 0..D, then interpolation; c has D + 1 words. */
static int residues_mod_p(const o2_poly *f, const o2_poly *g, const o2_plan *pl, uint32_t p, uint32_t *c) {
    scratch s;
    int rc = scratch_alloc(&s, f, g, pl);
    if (rc) return rc;
    int N = pl->D + 1;
    reduce_poly(f, pl->m_x, pl->m_y, p, s.fr, s.tmp);
    reduce_poly(g, pl->n_x, pl->n_y, p, s.gr, s.tmp);
    for (int x = 0; x < N && !rc; x++) rc = image_at(&s, pl, p, (uint32_t)x, &s.z[x]);
    if (!rc) lagrange(s.z, N, p, c, s.M, s.fact, s.ifact);
    scratch_free(&s);
    return rc;
}

/* ------------------------------------------------------------ thread pool */

typedef struct {
    int64_t next, ntasks;
    void (*fn)(void *, int64_t);
    void *arg;
} pool;

static void *pool_worker(void *a) {
    pool *P = (pool *)a;
    for (;;) {
        int64_t t = __atomic_fetch_add(&P->next, 1, __ATOMIC_RELAXED);
        if (t >= P->ntasks) break;
        P->fn(P->arg, t);
    }
    return NULL;
}

static void pool_run(int threads, int64_t ntasks, void (*fn)(void *, int64_t), void *arg) {
    pool P = {0, ntasks, fn, arg};
    if (threads < 1) threads = 1;
    if (threads > ntasks) threads = (int)(ntasks > 0 ? ntasks : 1);
    pthread_t *th = calloc((size_t)threads, sizeof(pthread_t));
    int started = 0;
    for (int t = 1; th && t < threads; t++)
        if (pthread_create(&th[started], NULL, pool_worker, &P) == 0) started++;
    pool_worker(&P);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
}

/* ------------------------------------------------------ Chinese remainders */

/* Per pair: the prefix products P_k = p_0 ... p_{k-1} (k = 0..K) and
 * inv_k = (P_k mod p_k)^-1 mod p_k. */
typedef struct {
    uint32_t *buf;  /* P_k at buf + off[k], len[k] limbs */
    int64_t *off;
    int *len;
    uint32_t *inv;
    uint32_t *half; /* floor(P_K / 2) */
    int nhalf;
} crt_table;

static void crt_free(crt_table *t) {
    free(t->buf); free(t->off); free(t->len); free(t->inv); free(t->half);
    memset(t, 0, sizeof(*t));
}

static int crt_prepare(int K, crt_table *t) {
    memset(t, 0, sizeof(*t));
    t->off = malloc(sizeof(int64_t) * (size_t)(K + 1));
    t->len = malloc(sizeof(int) * (size_t)(K + 1));
    t->inv = malloc(sizeof(uint32_t) * (size_t)(K > 0 ? K : 1));
    t->buf = malloc(sizeof(uint32_t) * ((size_t)(K + 1) * (K + 2) / 2 + (size_t)K + 2));
    t->half = malloc(sizeof(uint32_t) * (size_t)(K + 2));
    if (!t->off || !t->len || !t->inv || !t->buf || !t->half) {
        crt_free(t);
        return O2_ERR_NOMEM;
    }
    int64_t o = 0;
    t->off[0] = 0;
    t->buf[0] = 1;
    t->len[0] = 1;
    o = 1;
    for (int k = 1; k <= K; k++) {
        t->off[k] = o;
        t->len[k] = bn_mul_small(t->buf + t->off[k - 1], t->len[k - 1], o2_prime(k - 1), t->buf + o);
        o += t->len[k] + 1;
    }
    t->inv[0] = 1;
    for (int k = 1; k < K; k++) {
        uint32_t p = o2_prime(k);
        t->inv[k] = invm(bn_mod_small(t->buf + t->off[k], t->len[k], p), p);
    }
    /* half = P_K >> 1 */
    const uint32_t *P = t->buf + t->off[K];
    int n = t->len[K];
    for (int l = 0; l < n; l++) t->half[l] = (P[l] >> 1) | (l + 1 < n ? (P[l + 1] << 31) : 0);
    t->nhalf = bn_norm(t->half, n);
    return O2_OK;
}

/* One coefficient from its K residues r[k * stride]: x = r_0, then for each
 * next prime x += P_k * ((r_k - x) (P_k)^-1 mod p_k), which keeps x < P_{k+1}
 * and x = r_j mod p_j for every j <= k; finally the symmetric representative.
 * Writes out_limbs two's-complement limbs; returns 0, or O2_ERR_BOUND when
 * |value| needs more than bits + 1 bits. */
static int crt_one(const crt_table *t, int K, const uint32_t *r, int64_t stride, int bits, uint32_t *x,
                   uint32_t *mag, int out_limbs, uint32_t *out) {
    int nx = 0;
    x[0] = r[0];
    nx = bn_norm(x, 1);
    for (int k = 1; k < K; k++) {
        uint32_t p = o2_prime(k);
        uint32_t a = bn_mod_small(x, nx, p);
        uint32_t tk = mulm(subm(r[(int64_t)k * stride], a, p), t->inv[k], p);
        if (tk) nx = bn_addmul(x, nx, t->buf + t->off[k], t->len[k], tk);
    }
    int neg = bn_cmp(x, nx, t->half, t->nhalf) > 0 && O2_PLANT != 4;
    int nm;
    if (neg) {
        nm = bn_sub(t->buf + t->off[K], t->len[K], x, nx, mag);
    } else {
        memcpy(mag, x, sizeof(uint32_t) * (size_t)(nx ? nx : 1));
        nm = nx;
    }
    if (bn_bitlen(mag, nm) > bits + 1) return O2_ERR_BOUND;
    uint64_t carry = 1;
    for (int l = 0; l < out_limbs; l++) {
        uint32_t v = l < nm ? mag[l] : 0;
        if (neg) {
            uint64_t s = (uint64_t)(uint32_t)~v + carry;
            out[l] = (uint32_t)s;
            carry = s >> 32;
        } else {
            out[l] = v;
        }
    }
    return O2_OK;
}

/* ------------------------------------------------------------- the batch */

typedef struct {
    const o2_poly *f, *g;
    o2_plan pl;
    uint32_t *res; /* [K][D + 1] residues of R */
    crt_table crt;
    uint32_t *out;
    int status;
} pair_job;

typedef struct {
    pair_job *jobs;
    int32_t *task_pair, *task_k;
} batch_ctx;

static void set_status(pair_job *j, int rc) {
    if (rc) __atomic_store_n(&j->status, rc, __ATOMIC_RELAXED);
}

static void task_residues(void *a, int64_t t) {
    batch_ctx *B = (batch_ctx *)a;
    pair_job *j = &B->jobs[B->task_pair[t]];
    int k = B->task_k[t];
    int N = j->pl.D + 1;
    set_status(j, residues_mod_p(j->f, j->g, &j->pl, o2_prime(k), j->res + (int64_t)k * N));
}

static void task_crt_prepare(void *a, int64_t t) {
    batch_ctx *B = (batch_ctx *)a;
    pair_job *j = &B->jobs[t];
    if (j->pl.zero || j->status) return;
    set_status(j, crt_prepare(j->pl.nprimes, &j->crt));
}

#define CRT_BLOCK 32

static void task_crt(void *a, int64_t t) {
    batch_ctx *B = (batch_ctx *)a;
    pair_job *j = &B->jobs[B->task_pair[t]];
    if (j->status) return;
    int K = j->pl.nprimes, N = j->pl.D + 1, Lo = j->pl.out_limbs;
    uint32_t *x = malloc(sizeof(uint32_t) * (size_t)(K + 3));
    uint32_t *mag = malloc(sizeof(uint32_t) * (size_t)(K + 3));
    if (!x || !mag) {
        set_status(j, O2_ERR_NOMEM);
    } else {
        int c0 = B->task_k[t] * CRT_BLOCK;
        for (int c = c0; c < c0 + CRT_BLOCK && c < N; c++) {
            int rc = crt_one(&j->crt, K, j->res + c, N, j->pl.bits, x, mag, Lo, j->out + (int64_t)c * Lo);
            if (rc) { set_status(j, rc); break; }
        }
    }
    free(x);
    free(mag);
}

/* Resultants of n pairs.  out[i] must hold (plan.D + 1) * plan.out_limbs
 * words for o2_plan_pair(f + i, g + i) (one word when the plan says zero);
 * coefficient c of R_i is written at out[i] + c * out_limbs, c = 0..D, and
 * out_deg[i] receives deg R_i (-1 for R_i = 0).  Uses up to `threads`
 * threads.  Returns 0 or the first pair's error code. */
int o2_resultant_batch(int32_t n, const o2_poly *f, const o2_poly *g, int32_t threads, uint32_t *const *out,
                       int32_t *out_deg) {
    if (n < 0 || (n > 0 && (!f || !g || !out || !out_deg))) return O2_ERR_ARG;
    pthread_once(&g_primes_once, primes_init);
    pair_job *jobs = calloc((size_t)(n ? n : 1), sizeof(pair_job));
    if (!jobs) return O2_ERR_NOMEM;
    int rc = O2_OK;
    int64_t nres = 0, ncrt = 0;
    for (int i = 0; i < n && !rc; i++) {
        jobs[i].f = &f[i];
        jobs[i].g = &g[i];
        jobs[i].out = out[i];
        rc = o2_plan_pair(&f[i], &g[i], &jobs[i].pl);
        if (rc || jobs[i].pl.zero) continue;
        int N = jobs[i].pl.D + 1;
        jobs[i].res = malloc(sizeof(uint32_t) * (size_t)jobs[i].pl.nprimes * N);
        if (!jobs[i].res) rc = O2_ERR_NOMEM;
        nres += jobs[i].pl.nprimes;
        ncrt += (N + CRT_BLOCK - 1) / CRT_BLOCK;
    }
    batch_ctx B = {jobs, NULL, NULL};
    int64_t ntask = nres > ncrt ? nres : ncrt;
    if (!rc) {
        B.task_pair = malloc(sizeof(int32_t) * (size_t)(ntask ? ntask : 1));
        B.task_k = malloc(sizeof(int32_t) * (size_t)(ntask ? ntask : 1));
        if (!B.task_pair || !B.task_k) rc = O2_ERR_NOMEM;
    }
    if (!rc) {
        int64_t t = 0;
        for (int i = 0; i < n; i++)
            for (int k = 0; !jobs[i].pl.zero && k < jobs[i].pl.nprimes; k++) {
                B.task_pair[t] = i;
                B.task_k[t++] = k;
            }
        pool_run(threads, nres, task_residues, &B);
        pool_run(threads, n, task_crt_prepare, &B);
        t = 0;
        for (int i = 0; i < n; i++) {
            if (jobs[i].pl.zero) continue;
            int N = jobs[i].pl.D + 1;
            for (int b = 0; b < (N + CRT_BLOCK - 1) / CRT_BLOCK; b++) {
                B.task_pair[t] = i;
                B.task_k[t++] = b;
            }
        }
        pool_run(threads, ncrt, task_crt, &B);
        for (int i = 0; i < n && !rc; i++) rc = jobs[i].status;
    }
    for (int i = 0; i < n; i++) {
        if (!rc) {
            pair_job *j = &jobs[i];
            int d = -1;
            if (j->pl.zero) {
                j->out[0] = 0;
            } else {
                int Lo = j->pl.out_limbs;
                for (int c = j->pl.D; c >= 0 && d < 0; c--)
                    for (int l = 0; l < Lo; l++)
                        if (j->out[(int64_t)c * Lo + l]) { d = c; break; }
            }
            out_deg[i] = d;
        }
        free(jobs[i].res);
        crt_free(&jobs[i].crt);
    }
    free(B.task_pair);
    free(B.task_k);
    free(jobs);
    return rc;
}

/* --------------------------------------------------- entry points for pins */

/* One image det S(x) mod p (any prime p < 2^31 with p > 2): `how` = 0 picks
 * as the batch does (Euclid when both leading coefficients survive, else the
 * Sylvester matrix), 1 forces the Sylvester matrix, 2 forces Euclid and
 * returns O2_ERR_ARG through *rc when a leading coefficient vanishes. */
uint32_t o2_image(const o2_poly *f, const o2_poly *g, uint32_t p, uint32_t x, int32_t how, int32_t *rc) {
    o2_plan pl;
    int e = o2_plan_pair(f, g, &pl);
    uint32_t v = 0;
    if (!e && pl.zero) { *rc = O2_OK; return 0; }
    if (e) { *rc = e; return 0; }
    pl.D = 0; /* only the point x is needed */
    scratch s;
    e = scratch_alloc(&s, f, g, &pl);
    if (e) { *rc = e; return 0; }
    reduce_poly(f, pl.m_x, pl.m_y, p, s.fr, s.tmp);
    reduce_poly(g, pl.n_x, pl.n_y, p, s.gr, s.tmp);
    x %= p;
    eval_rows(s.fr, pl.m_x, pl.m_y, x, p, s.F);
    eval_rows(s.gr, pl.n_x, pl.n_y, x, p, s.G);
    int lucky = s.F[pl.m_y] && s.G[pl.n_y];
    if (how == 2 && !lucky) {
        e = O2_ERR_ARG;
    } else if (how == 0) {
        e = image_at(&s, &pl, p, x, &v);
    } else if (how == 1) {
        size_t r = (size_t)(pl.m_y + pl.n_y);
        s.syl = malloc(sizeof(uint32_t) * (r ? r * r : 1));
        if (!s.syl) e = O2_ERR_NOMEM;
        else v = res_sylvester(s.F, pl.m_y, s.G, pl.n_y, p, s.syl);
    } else {
        memcpy(s.A, s.F, sizeof(uint32_t) * (size_t)(pl.m_y + 1));
        memcpy(s.B, s.G, sizeof(uint32_t) * (size_t)(pl.n_y + 1));
        v = res_euclid(s.A, pl.m_y, s.B, pl.n_y, p);
    }
    scratch_free(&s);
    *rc = e;
    return v;
}

/* R mod p for one pair and one prime p (D + 1 > p not allowed): coefficients
 * 0..plan.D into c. */
int o2_residues(const o2_poly *f, const o2_poly *g, uint32_t p, uint32_t *c) {
    o2_plan pl;
    int e = o2_plan_pair(f, g, &pl);
    if (e) return e;
    if (pl.zero) { c[0] = 0; return O2_OK; }
    if ((uint32_t)pl.D + 1 >= p) return O2_ERR_ARG;
    return residues_mod_p(f, g, &pl, p, c);
}

/* Chinese remaindering alone, for pins: ncoef coefficients from residues
 * r[k * ncoef + c] modulo the first K table primes, into out[c * out_limbs]
 * (two's complement, symmetric range); `bits` as in the plan. */
int o2_crt(int32_t K, int32_t ncoef, const uint32_t *r, int32_t bits, int32_t out_limbs, uint32_t *out) {
    if (K < 1 || K > O2_MAX_PRIMES || ncoef < 0 || out_limbs < (31 * K + 31) / 32) return O2_ERR_ARG;
    pthread_once(&g_primes_once, primes_init);
    crt_table t;
    int rc = crt_prepare(K, &t);
    if (rc) return rc;
    uint32_t *x = malloc(sizeof(uint32_t) * (size_t)(K + 3));
    uint32_t *mag = malloc(sizeof(uint32_t) * (size_t)(K + 3));
    if (!x || !mag) rc = O2_ERR_NOMEM;
    for (int c = 0; c < ncoef && !rc; c++)
        rc = crt_one(&t, K, r + c, ncoef, bits, x, mag, out_limbs, out + (int64_t)c * out_limbs);
    free(x);
    free(mag);
    crt_free(&t);
    return rc;
}
