/*
 * CPU oracle for the RSA-exponentiation pseudorandom generator of
 * Datephanyawat & Beale, "A class of scalable parallel and vectorizable
 * pseudorandom number generators based on non-cryptographic RSA
 * exponentiation ciphers" (arXiv:1811.11629).
 *
 * TEST INFRASTRUCTURE. This file is the plain, slow, obviously correct
 * definition that the GPU library is checked against. Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it. It shares
 * no source with the GPU library (no headers, helpers or constant tables);
 * the only thing both sides share is the seeded input generator module,
 * which holds none of the method's arithmetic.
 *
 * Everything is done in plain C with unsigned __int128 (the direct route) and
 * with the paper's native 64-bit route (Schrage decomposition + CRT, Eq.
 * algorithm1 of Sec. V). The checked generator runs both routes and reports a
 * mismatch as an error.
 *
 * Parity status of each function (what pins it is in the test suite):
 *   or_mulmod / or_powmod        pinned: primitive-root orders, RSA inverse
 *                                round trip, permutation of Z_n (brute force)
 *   or_is_prime                  pinned: prime counts of Sec. V, sieve, and
 *                                Q = 2^63-25 being the largest prime < 2^63
 *   or_skip_next_*               pinned: closed form s_k = s_0 a^k mod Q and
 *                                the period structure of Sec. IV (tiny Q)
 *   or_crt_encrypt               pinned: CRT residues, Garner reconstruction
 *   or_crt_encrypt2 / or_crt_exponent
 *                                pinned: residue-wise powers, m^E mod n with
 *                                E from a Python CRT, permutation of Z_n
 *   or_unit                      pinned: exact-rational rounding of the two
 *                                IEEE conversions and the division
 *   or_unit_exact                pinned: Python's correctly rounded
 *                                float(Fraction(c, n)), ties built exactly
 *   or_generate (sequence)       pinned by the closed form of Eq. pseudoskip
 *                                on tiny Q and by the two routes agreeing
 *   or_params_from_seed          pinned: SplitMix64 published test values
 *                                and the parameter rules re-checked by MR
 *   or_generate_vector           pinned: equals the per-instance streams of
 *                                or_generate interleaved k-major
 *   or_digit_of_unit             pinned: exact-rational floor(r d) for
 *                                power-of-two and decimal d, boundaries
 *   or_histogram                 pinned: tuple counts rebuilt from the
 *                                generated sequence, total = floor(N / D)
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

/* Q = 2^63 - 25, the skip modulus of Sec. V. */
#define OR_Q ((uint64_t)0x7FFFFFFFFFFFFFE7ULL)

/* Error codes of the oracle (its own; unrelated to the library's). */
#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_ROUTE_MISMATCH (-2)

uint64_t or_q_default(void) { return OR_Q; }

/* ------------------------------------------------------------------ */
/* Modular arithmetic (Sec. I, Sec. III)                                */
/* ------------------------------------------------------------------ */

/* (a * b) mod m with a 128-bit product; m > 0. */
uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a * (u128)b) % (u128)m);
}

/* (a + b) mod m for a, b < m; computed in 128 bits so no carry is lost. */
uint64_t or_addmod(uint64_t a, uint64_t b, uint64_t m)
{
    return (uint64_t)(((u128)a + (u128)b) % (u128)m);
}

/* b^e mod m by repeated squaring and multiplying (Sec. I: fewer than
 * 2 log2 e modular multiplications). Direct route, 128-bit products. */
uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1)
            r = or_mulmod(r, b, m);
        b = or_mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

/* b^e mod m for m < 2^32 using only native 64-bit products: the route of
 * the CRT steps of Eq. algorithm1 ("fast native 64-bit arithmetic"). */
static uint64_t or_powmod_native32(uint64_t b, uint64_t e, uint64_t m)
{
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1)
            r = (r * b) % m;
        b = (b * b) % m;
        e >>= 1;
    }
    return r;
}

uint64_t or_gcd(uint64_t a, uint64_t b)
{
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* a^{-1} mod m by the extended Euclidean algorithm (Sec. III, Eq. RSAd);
 * returns 0 when gcd(a, m) != 1. */
uint64_t or_invmod(uint64_t a, uint64_t m)
{
    __int128 t0 = 0, t1 = 1, r0 = (__int128)m, r1 = (__int128)(a % m);
    while (r1 != 0) {
        __int128 qt = r0 / r1, tmp;
        tmp = r0 - qt * r1; r0 = r1; r1 = tmp;
        tmp = t0 - qt * t1; t0 = t1; t1 = tmp;
    }
    if (r0 != 1)
        return 0;
    if (t0 < 0)
        t0 += (__int128)m;
    return (uint64_t)t0;
}

/* ------------------------------------------------------------------ */
/* Primality (Sec. V): trial division by small primes, then Rabin-Miller */
/* ------------------------------------------------------------------ */

static const uint64_t OR_SMALL_PRIMES[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};

/* One Rabin-Miller round: with n - 1 = 2^u t (t odd), n passes base g when
 * g^t = 1 or g^(2^j t) = n - 1 for some 0 <= j < u. */
static int or_rabin_miller_base(uint64_t n, uint64_t g)
{
    uint64_t t = n - 1;
    int u = 0;
    while ((t & 1) == 0) {
        t >>= 1;
        u++;
    }
    uint64_t x = or_powmod(g, t, n);
    if (x == 1 || x == n - 1)
        return 1;
    for (int j = 1; j < u; j++) {
        x = or_mulmod(x, x, n);
        if (x == n - 1)
            return 1;
    }
    return 0;
}

/* Deterministic primality for any 64-bit n: the five smallest prime bases
 * are conclusive below 2^32 and the twelve smallest below 2^64 (Sec. V). */
int or_is_prime(uint64_t n)
{
    if (n < 2)
        return 0;
    for (int i = 0; i < 12; i++) {
        if (n == OR_SMALL_PRIMES[i])
            return 1;
        if (n % OR_SMALL_PRIMES[i] == 0)
            return 0;
    }
    if (n < 37 * 37)
        return 1;
    int bases = (n < ((uint64_t)1 << 32)) ? 5 : 12;
    for (int i = 0; i < bases; i++)
        if (!or_rabin_miller_base(n, OR_SMALL_PRIMES[i]))
            return 0;
    return 1;
}

/* Counts primes and safe primes p ((p-1)/2 prime) in [lo, hi). Used to pin
 * the primality test against the counts printed in Sec. V. */
void or_count_primes(uint64_t lo, uint64_t hi, uint64_t *primes, uint64_t *safe)
{
    uint64_t np = 0, ns = 0;
    int64_t start = (int64_t)(lo | 1), stop = (int64_t)hi;
#pragma omp parallel for schedule(dynamic, 65536) reduction(+ : np, ns)
    for (int64_t x = start; x < stop; x += 2) {
        if (or_is_prime((uint64_t)x)) {
            np++;
            if (or_is_prime(((uint64_t)x - 1) / 2))
                ns++;
        }
    }
    if (lo <= 2 && hi > 2)
        np++;
    *primes = np;
    *safe = ns;
}

/* ------------------------------------------------------------------ */
/* Skip generator (Sec. IV, Eq. congruentialgenerator1; Sec. V)         */
/* ------------------------------------------------------------------ */

/* s' = a s mod Q with a 128-bit product. */
uint64_t or_skip_next_direct(uint64_t s, uint64_t a, uint64_t Q)
{
    return or_mulmod(a, s, Q);
}

/* s' = a s mod Q by the decomposition of Eq. restrictedprimitiveroots with
 * q1 = floor(Q/a), q2 = Q mod a (steps WH1-WH3 of Eq. algorithm1); only
 * native 64-bit operations. Valid when q2 < q1. The subtraction in WH3 is
 * done without a negative intermediate. */
uint64_t or_skip_next_schrage(uint64_t s, uint64_t a, uint64_t Q)
{
    uint64_t q1 = Q / a, q2 = Q % a;
    uint64_t s1 = a * (s % q1);
    uint64_t s2 = q2 * (s / q1);
    return (s1 >= s2) ? (s1 - s2) : (s1 + (Q - s2));
}

/* s_0 a^k mod Q, the jump of Eq. pseudoskip. */
uint64_t or_skip_jump(uint64_t s0, uint64_t a, uint64_t k, uint64_t Q)
{
    return or_mulmod(s0, or_powmod(a, k, Q), Q);
}

/* Skip of substream gamma out of Mv (Sec. VI): s0 a^(gamma floor((Q-1)/Mv)). */
uint64_t or_split_s0(uint64_t s0, uint64_t a, uint64_t Q, uint64_t Mv, uint64_t gamma)
{
    u128 k = (u128)gamma * (u128)((Q - 1) / Mv);
    /* k < Q - 1 + 1 fits in 64 bits since gamma < Mv. */
    return or_skip_jump(s0, a, (uint64_t)k, Q);
}

/* ------------------------------------------------------------------ */
/* Encryption (Sec. III, Eq. encrypt and Eq. CRTimplementation)         */
/* ------------------------------------------------------------------ */

/* c = m^e mod n, the direct route. */
uint64_t or_encrypt_direct(uint64_t m, uint64_t e, uint64_t n)
{
    return or_powmod(m, e, n);
}

/* c from the residues m_p, m_q by CRT and Garner's formula (steps
 * CodeExponentiationStep1-3 of Eq. algorithm1): c_p = m_p^ep mod p,
 * c_q = m_q^eq mod q, c = (((c_p - c_q) q^{-1} mod p) mod p) q + c_q, with
 * ep = eq = e for the ordinary generator. The difference is formed as
 * (c_p + p - (c_q mod p)) so it never goes negative (c_q can exceed p when
 * q > p). */
uint64_t or_crt_encrypt2(uint64_t mp, uint64_t mq, uint64_t p, uint64_t q, uint64_t ep,
                         uint64_t eq, uint64_t qinv_p)
{
    uint64_t cp = or_powmod_native32(mp, ep, p);
    uint64_t cq = or_powmod_native32(mq, eq, q);
    uint64_t diff = (cp + p - (cq % p)) % p;
    uint64_t h = (diff * qinv_p) % p;
    return h * q + cq;
}

uint64_t or_crt_encrypt(uint64_t mp, uint64_t mq, uint64_t p, uint64_t q, uint64_t e,
                        uint64_t qinv_p)
{
    return or_crt_encrypt2(mp, mq, p, q, e, e, qinv_p);
}

/* The single exponent of CRT exponents (the paper's note on large exponents,
 * Sec. V): E with E = ep (mod p-1) and E = eq (mod q-1), 0 <= E <
 * lcm(p-1, q-1), by the CRT for the moduli p-1 and q-1 (not coprime: a
 * solution exists iff ep = eq mod gcd(p-1, q-1)). Returns 0 when there is
 * none (E itself is never 0: E = ep >= 1 mod p-1). */
uint64_t or_crt_exponent(uint64_t p, uint64_t q, uint64_t ep, uint64_t eq)
{
    const uint64_t a = p - 1, b = q - 1;
    const uint64_t g = or_gcd(a, b);
    const uint64_t ra = ep % a, rb = eq % b;
    const uint64_t diff = (rb + b - (ra % b)) % b; /* eq - ep mod b */
    if (diff % g != 0)
        return 0;
    /* E = ra + a t with a t = diff (mod b): t = (diff / g) (a / g)^-1 mod (b / g) */
    const uint64_t bg = b / g;
    const uint64_t inv = (bg == 1) ? 0 : or_invmod((a / g) % bg, bg);
    const uint64_t t = (bg == 1) ? 0 : (uint64_t)(((u128)((diff / g) % bg) * inv) % bg);
    return ra + a * t; /* < a (b / g) = lcm(a, b) < 2^64 */
}

/* ------------------------------------------------------------------ */
/* Output (Eq. CodeFloatingPointStep)                                   */
/* ------------------------------------------------------------------ */

/* r = c / n as IEEE doubles: both integers are converted to double with
 * round-to-nearest-even and divided. Because n > 2^53 the quotient can round
 * up to 1.0 (Sec. V); that value is replaced by the largest double below 1. */
double or_unit(uint64_t c, uint64_t n)
{
    volatile double dc = (double)c;
    volatile double dn = (double)n;
    double r = dc / dn;
    if (r >= 1.0)
        r = 0x1.fffffffffffffp-1;
    return r;
}

/* The other reading of the division: r = RN(c / n), the exact rational c/n
 * rounded once to the nearest double (ties to even), with the same 1.0
 * guard. Long division, one bit at a time: the quotient bits of c/n < 1 are
 * produced until 53 significant bits and the next (round) bit are known; the
 * remainder left over decides the ties (sticky). */
double or_unit_exact(uint64_t c, uint64_t n)
{
    if (c == 0)
        return 0.0;
    u128 rem = c;
    int pos = 0, nbits = 0;
    uint64_t sig = 0;
    while (nbits < 54) {
        rem <<= 1;
        pos++;
        const int b = rem >= n;
        if (b)
            rem -= n;
        if (nbits > 0 || b) {
            sig = (sig << 1) | (uint64_t)b;
            nbits++;
        }
    }
    /* sig: 53 significand bits and the round bit (weight 2^-pos) */
    uint64_t m = sig >> 1;
    const int round_bit = (int)(sig & 1), sticky = rem != 0;
    if (round_bit && (sticky || (m & 1)))
        m++;
    double r = ldexp((double)m, -(pos - 1));
    if (r >= 1.0)
        r = 0x1.fffffffffffffp-1;
    return r;
}

/* ------------------------------------------------------------------ */
/* One generator instance (Sec. IV state {n, e, Q, a} + {m, s})         */
/* ------------------------------------------------------------------ */

/* eq: the exponent of the q residue (CRT exponents); 0 means eq = e. */
typedef struct {
    uint64_t p, q, e, a, Q, eq;
} or_params;

enum { OR_ROUTE_CHECKED = 0, OR_ROUTE_PAPER = 1, OR_ROUTE_DIRECT = 2 };

/*
 * Emits N outputs of one instance starting from state (m, s) and leaves the
 * state after the last output in (*m, *s). Output k (k = 1..N) is
 *     s_k = a s_{k-1} mod Q,  m_k = (m_{k-1} + s_k) mod n,
 *     c_k = m_k^e mod n,      r_k = c_k / n   (with the 1.0 guard),
 * i.e. the first output comes from m_1 = m_0 + a s_0 (Eq. pseudoskip sums
 * from j = 1). c_out / r_out may be NULL.
 *
 * Routes: PAPER follows Eq. algorithm1 exactly (Schrage skip, residues m_p,
 * m_q, CRT + Garner); DIRECT uses 128-bit products on m itself; CHECKED runs
 * both and returns OR_ERR_ROUTE_MISMATCH at the first disagreement.
 */
int or_generate(const or_params *P, uint64_t *m_io, uint64_t *s_io, uint64_t N,
                uint64_t *c_out, double *r_out, int route)
{
    const uint64_t p = P->p, q = P->q, e = P->e, a = P->a, Q = P->Q;
    const uint64_t eq = P->eq ? P->eq : e;
    const uint64_t n = p * q;
    uint64_t m = *m_io, s = *s_io;
    uint64_t mp = m % p, mq = m % q;
    const uint64_t qinv_p = or_invmod(q % p, p);
    const int schrage_ok = (Q % a) < (Q / a);
    /* The direct route needs one exponent: e itself, or the CRT exponent. */
    const uint64_t E = (eq == e) ? e : or_crt_exponent(p, q, e, eq);
    if (p < 2 || q < 2 || a < 1 || a >= Q || m >= n || s == 0 || s >= Q)
        return OR_ERR_ARG;
    if (route != OR_ROUTE_DIRECT && (p >= ((uint64_t)1 << 32) || q >= ((uint64_t)1 << 32) || !schrage_ok || qinv_p == 0))
        return OR_ERR_ARG;
    if (route == OR_ROUTE_DIRECT && E == 0)
        return OR_ERR_ARG;

    for (uint64_t k = 0; k < N; k++) {
        uint64_t c;
        if (route == OR_ROUTE_PAPER) {
            s = or_skip_next_schrage(s, a, Q);
            mp = (mp + s) % p;
            mq = (mq + s) % q;
            c = or_crt_encrypt2(mp, mq, p, q, e, eq, qinv_p);
        } else if (route == OR_ROUTE_DIRECT) {
            s = or_skip_next_direct(s, a, Q);
            m = or_addmod(m, s % n, n);
            c = or_encrypt_direct(m, E, n);
        } else {
            uint64_t s_direct = or_skip_next_direct(s, a, Q);
            uint64_t s_paper = or_skip_next_schrage(s, a, Q);
            if (s_direct != s_paper)
                return OR_ERR_ROUTE_MISMATCH;
            s = s_direct;
            m = or_addmod(m, s % n, n);
            mp = (mp + s) % p;
            mq = (mq + s) % q;
            if (m % p != mp || m % q != mq)
                return OR_ERR_ROUTE_MISMATCH;
            uint64_t c_paper = or_crt_encrypt2(mp, mq, p, q, e, eq, qinv_p);
            if (E != 0 && or_encrypt_direct(m, E, n) != c_paper)
                return OR_ERR_ROUTE_MISMATCH;
            c = c_paper;
        }
        if (c_out)
            c_out[k] = c;
        if (r_out)
            r_out[k] = or_unit(c, n);
    }
    if (route == OR_ROUTE_PAPER) {
        /* Recover m from its residues with Garner's formula (Sec. III). */
        uint64_t diff = (mp + p - (mq % p)) % p;
        m = ((diff * qinv_p) % p) * q + mq;
    }
    *m_io = m;
    *s_io = s;
    return OR_OK;
}

/*
 * Advances the state by k outputs without encrypting: k steps of
 * s <- a s mod Q, m <- (m + s) mod n (Sec. IV). This is the summation of
 * Eq. pseudoskip carried out term by term.
 */
int or_seek(const or_params *P, uint64_t *m_io, uint64_t *s_io, uint64_t k)
{
    const uint64_t n = P->p * P->q;
    uint64_t m = *m_io, s = *s_io;
    if (m >= n || s == 0 || s >= P->Q)
        return OR_ERR_ARG;
    for (uint64_t i = 0; i < k; i++) {
        s = or_skip_next_direct(s, P->a, P->Q);
        m = or_addmod(m, s % n, n);
    }
    *m_io = m;
    *s_io = s;
    return OR_OK;
}

/*
 * or_seek over all host cores: the message advances by the sum of the k next
 * skips (Sec. IV, Eq. pseudoskip), and the sum splits into consecutive
 * ranges; the range starting after j skips begins from s a^j mod Q (the
 * skip's jump-ahead, Eq. congruentialgenerator1), so every thread walks its
 * own range with the skip recurrence and the partial sums are added mod n.
 */
int or_seek_parallel(const or_params *P, uint64_t *m_io, uint64_t *s_io, uint64_t k)
{
    enum { MAXT = 1024 };
    const uint64_t n = P->p * P->q, a = P->a, Q = P->Q;
    const uint64_t s0 = *s_io;
    if (*m_io >= n || s0 == 0 || s0 >= Q)
        return OR_ERR_ARG;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    if (nt > MAXT)
        nt = MAXT;
    uint64_t part[MAXT];
    const uint64_t per = (k + (uint64_t)nt - 1) / (uint64_t)nt;
#pragma omp parallel for schedule(static, 1) num_threads(nt)
    for (int t = 0; t < nt; t++) {
        const uint64_t lo = (uint64_t)t * per;
        const uint64_t hi = (lo + per < k) ? lo + per : k;
        uint64_t s = or_mulmod(s0, or_powmod(a, lo, Q), Q);
        uint64_t sum = 0;
        for (uint64_t j = lo; j < hi; j++) {
            s = or_skip_next_direct(s, a, Q);
            sum = or_addmod(sum, s % n, n);
        }
        part[t] = sum;
    }
    uint64_t m = *m_io;
    for (int t = 0; t < nt; t++)
        m = or_addmod(m, part[t], n);
    *m_io = m;
    *s_io = or_mulmod(s0, or_powmod(a, k, Q), Q);
    return OR_OK;
}

/*
 * Sampled outputs of one instance: for the increasing 1-based output indices
 * ks[0] < ks[1] < ... < ks[nk-1], c_out[j] / r_out[j] receive c_k, r_k with
 * k = ks[j]. The state is advanced by Sec. IV's sums (or_seek) between the
 * samples and each sample is encrypted by the direct route. (*m_io, *s_io)
 * end at output ks[nk-1].
 */
int or_sample(const or_params *P, uint64_t *m_io, uint64_t *s_io, const uint64_t *ks,
              uint64_t nk, uint64_t *c_out, double *r_out)
{
    const uint64_t n = P->p * P->q;
    uint64_t done = 0;
    for (uint64_t j = 0; j < nk; j++) {
        if (ks[j] <= done)
            return OR_ERR_ARG;
        int rc = or_seek(P, m_io, s_io, ks[j] - done);
        if (rc != OR_OK)
            return rc;
        done = ks[j];
        uint64_t c = or_encrypt_direct(*m_io, P->e, n);
        if (c_out)
            c_out[j] = c;
        if (r_out)
            r_out[j] = or_unit(c, n);
    }
    return OR_OK;
}

/* or_sample over many instances in parallel: instance i samples the nk[i]
 * indices at ks + koff[i] and writes at c_out/r_out + koff[i]. */
int or_sample_many(uint64_t count, const uint64_t *p, const uint64_t *q, const uint64_t *e,
                   const uint64_t *a, uint64_t Q, uint64_t *m, uint64_t *s, const uint64_t *ks,
                   const uint64_t *koff, const uint64_t *nk, uint64_t *c_out, double *r_out)
{
    int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        or_params P = {p[i], q[i], e[i], a[i], Q, 0};
        int rc = or_sample(&P, &m[i], &s[i], ks + koff[i], nk[i], c_out ? c_out + koff[i] : NULL,
                           r_out ? r_out + koff[i] : NULL);
        if (rc != OR_OK) {
#pragma omp critical
            if (err == OR_OK)
                err = rc;
        }
    }
    return err;
}

/* r[i] = or_unit_exact(c[i], n) for i < count. */
void or_unit_exact_many(const uint64_t *c, uint64_t n, double *r, uint64_t count)
{
    for (uint64_t i = 0; i < count; i++)
        r[i] = or_unit_exact(c[i], n);
}

/* r[i] = or_unit(c[i], n) for i < count. */
void or_unit_many(const uint64_t *c, uint64_t n, double *r, uint64_t count)
{
    for (uint64_t i = 0; i < count; i++)
        r[i] = or_unit(c[i], n);
}

/*
 * Many independent instances (parameterization, Sec. VI), one output region
 * per instance: instance i writes counts[i] values at offsets[i] of c_out /
 * r_out (either may be NULL) and has its state (m[i], s[i]) advanced.
 * Instances run in parallel over the host cores with OpenMP, as the paper's
 * CPU implementation does. Returns the first error seen, else OR_OK.
 */
int or_generate_many(uint64_t count, const uint64_t *p, const uint64_t *q, const uint64_t *e,
                     const uint64_t *a, uint64_t Q, uint64_t *m, uint64_t *s,
                     const uint64_t *counts, const uint64_t *offsets, uint64_t *c_out,
                     double *r_out, int route)
{
    int err = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        or_params P = {p[i], q[i], e[i], a[i], Q, 0};
        int rc = or_generate(&P, &m[i], &s[i], counts[i], c_out ? c_out + offsets[i] : NULL,
                             r_out ? r_out + offsets[i] : NULL, route);
        if (rc != OR_OK) {
#pragma omp critical
            if (err == OR_OK)
                err = rc;
        }
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* Frequency and serial test histograms (Sec. VII)                      */
/* ------------------------------------------------------------------ */

/* floor(r d) for a double r in [0, 1) and an integer d < 2^32, exactly: r is
 * f 2^x with f in [1/2, 1) holding at most 53 significant bits, so
 * r = M / 2^(53 - x) with the integer M = f 2^53, and the floor of r d is the
 * integer quotient (M d) >> (53 - x). */
uint64_t or_digit_of_unit(double r, uint64_t d)
{
    if (r == 0.0)
        return 0;
    int x;
    const double f = frexp(r, &x);
    const uint64_t M = (uint64_t)ldexp(f, 53);
    const int sh = 53 - x;
    if (sh >= 128)
        return 0;
    return (uint64_t)(((u128)M * d) >> sh);
}

/*
 * The histogram of the one-dimensional frequency test (D = 1) and the
 * D-dimensional serial test (Sec. VII) over the next N outputs of one
 * instance: the outputs are cut into non-overlapping D-tuples of consecutive
 * outputs, each tuple (x_1, ..., x_D) adds one to
 * hist[digit(x_1) + digit(x_2) d + ... + digit(x_D) d^(D-1)], with
 * digit = floor(r d) of the float output (source 0) or c mod d of the
 * ciphertext (source 1). Outputs after the last whole tuple are generated
 * (the state advances by N) but not counted. hist has d^D entries and is
 * added to.
 */
int or_histogram(const or_params *P, uint64_t *m_io, uint64_t *s_io, uint64_t N, uint64_t D,
                 uint64_t d, int source, int route, uint64_t *hist)
{
    enum { BLK = 4096 };
    uint64_t c[BLK];
    double r[BLK];
    uint64_t bin = 0, w = 1, filled = 0;
    if (D < 1 || d < 2)
        return OR_ERR_ARG;
    for (uint64_t done = 0; done < N;) {
        const uint64_t k = (N - done < BLK) ? N - done : BLK;
        const int rc = or_generate(P, m_io, s_io, k, c, r, route);
        if (rc != OR_OK)
            return rc;
        for (uint64_t i = 0; i < k; i++) {
            const uint64_t g = (source == 0) ? or_digit_of_unit(r[i], d) : c[i] % d;
            bin += g * w;
            w *= d;
            if (++filled == D) {
                hist[bin]++;
                bin = 0;
                w = 1;
                filled = 0;
            }
        }
        done += k;
    }
    return OR_OK;
}

/* or_histogram over many instances (OpenMP over instances, one private
 * histogram per thread, summed at the end); m[i], s[i] are advanced. */
int or_histogram_many(uint64_t count, const uint64_t *p, const uint64_t *q, const uint64_t *e,
                      const uint64_t *a, uint64_t Q, uint64_t *m, uint64_t *s,
                      const uint64_t *counts, uint64_t D, uint64_t d, int source, int route,
                      uint64_t *hist)
{
    uint64_t bins = 1;
    for (uint64_t i = 0; i < D; i++)
        bins *= d;
    int err = OR_OK;
#pragma omp parallel
    {
        uint64_t *mine = (uint64_t *)calloc(bins, sizeof(uint64_t));
        if (!mine) {
#pragma omp critical
            err = OR_ERR_ARG;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < (int64_t)count; i++) {
            if (!mine)
                continue;
            or_params P = {p[i], q[i], e[i], a[i], Q, 0};
            const int rc = or_histogram(&P, &m[i], &s[i], counts[i], D, d, source, route, mine);
            if (rc != OR_OK) {
#pragma omp critical
                if (err == OR_OK)
                    err = rc;
            }
        }
        if (mine) {
#pragma omp critical
            for (uint64_t b = 0; b < bins; b++)
                hist[b] += mine[b];
            free(mine);
        }
    }
    return err;
}

/*
 * The vectorised call of Sec. VI (Eq. vectorize), written out: the Mv
 * instances' skips, messages, ciphertexts and reals are updated together, one
 * vector per step, and step k (k = 1..N) writes element gamma of its vector at
 * (k - 1) Mv + gamma of c_out / r_out (either may be NULL). Instance gamma has
 * parameters (p, q, e, a)[gamma] and state (m, s)[gamma], advanced in place.
 */
int or_generate_vector(uint64_t Mv, const uint64_t *p, const uint64_t *q, const uint64_t *e,
                       const uint64_t *a, uint64_t Q, uint64_t *m, uint64_t *s, uint64_t N,
                       uint64_t *c_out, double *r_out)
{
    for (uint64_t k = 0; k < N; k++) {
        for (uint64_t g = 0; g < Mv; g++) {
            const uint64_t n = p[g] * q[g];
            if (p[g] < 2 || q[g] < 2 || a[g] < 1 || a[g] >= Q || m[g] >= n || s[g] == 0 ||
                s[g] >= Q)
                return OR_ERR_ARG;
            s[g] = or_skip_next_direct(s[g], a[g], Q);
            m[g] = or_addmod(m[g], s[g] % n, n);
            const uint64_t c = or_encrypt_direct(m[g], e[g], n);
            if (c_out)
                c_out[k * Mv + g] = c;
            if (r_out)
                r_out[k * Mv + g] = or_unit(c, n);
        }
    }
    return OR_OK;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Seeded instance parameters                                            */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the state advances by the
 * golden-ratio increment and each output is the state passed through the
 * published 64-bit finalizer. */
uint64_t or_splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

enum { OR_E_SMALLEST = 0, OR_E_UNIFORM = 1, OR_E_AT_LEAST = 2 };

/*
 * Instance parameters from one 64-bit seed, by the rule the workloads use:
 * draws x come from SplitMix64 started at `seed`; a prime candidate is the
 * high half of a draw with its top and bottom bits set (a 32-bit odd number
 * in [2^31, 2^32)); p is the first prime candidate and q the next prime
 * candidate different from p. The exponent follows `e_rule`:
 *   SMALLEST  the smallest odd e >= 3 with gcd(e, (p-1)(q-1)) = 1;
 *   AT_LEAST  the smallest such odd e >= e_lo;
 *   UNIFORM   draws e = e_lo + 2 (x mod ((e_hi - e_lo)/2 + 1)) until
 *             gcd(e, (p-1)(q-1)) = 1 (e_lo odd).
 * Finally the message seed is the next draw; the instance starts at
 * m_0 = seed mod n, s_0 = 1.
 */
int or_params_from_seed(uint64_t seed, int e_rule, uint64_t e_lo, uint64_t e_hi, uint64_t *p_out,
                        uint64_t *q_out, uint64_t *e_out, uint64_t *msg_seed_out)
{
    uint64_t st = seed, p, q, e;
    do {
        p = (or_splitmix64_next(&st) >> 32) | 0x80000001ULL;
    } while (!or_is_prime(p));
    do {
        q = (or_splitmix64_next(&st) >> 32) | 0x80000001ULL;
    } while (q == p || !or_is_prime(q));
    const uint64_t phi = (p - 1) * (q - 1);
    if (e_rule == OR_E_SMALLEST || e_rule == OR_E_AT_LEAST) {
        e = (e_rule == OR_E_SMALLEST) ? 3 : (e_lo | 1);
        while (or_gcd(e, phi) != 1)
            e += 2;
    } else if (e_rule == OR_E_UNIFORM) {
        if ((e_lo & 1) == 0 || e_hi < e_lo)
            return OR_ERR_ARG;
        const uint64_t span = (e_hi - e_lo) / 2 + 1;
        do {
            e = e_lo + 2 * (or_splitmix64_next(&st) % span);
        } while (or_gcd(e, phi) != 1);
    } else {
        return OR_ERR_ARG;
    }
    *p_out = p;
    *q_out = q;
    *e_out = e;
    *msg_seed_out = or_splitmix64_next(&st);
    return OR_OK;
}
