// Host-side number theory for instance setup (arXiv:1811.11629 Sec. III-V).
#include "host_params.hpp"

#include <cmath>

#include "../../include/rsaprng.h"

namespace rsaprng {

// Root list: the L'Ecuyer-Blouin-Couture recommendation, the eight Sezgin &
// Sezgin multipliers that are primitive roots mod Q (3163786287 from the same
// list is a quadratic residue and is left out), the five smallest primitive
// roots mod Q (Sec. VII's weakened-generator tests), and 1: with a = 1 the
// skip stays s_0, the unit (s_0 = 1) or constant skip of Sec. IV.
const u64 kRoots[kNumRoots] = {
    2307085864ULL, 3157107955ULL, 3200261722ULL, 3211103532ULL, 3338736601ULL,
    3423977237ULL, 3465965455ULL, 3474009732ULL, 3512424704ULL,
    3ULL,          6ULL,          7ULL,          10ULL,         11ULL,
    1ULL,
};

int root_index(u64 a)
{
    for (int i = 0; i < kNumRoots; i++)
        if (kRoots[i] == a)
            return i;
    return -1;
}

u64 mulmod(u64 a, u64 b, u64 m) { return (u64)(((u128)a * b) % m); }

u64 powmod(u64 b, u64 e, u64 m)
{
    u64 acc = 1 % m;
    b %= m;
    for (int bit = 63; bit >= 0; bit--) {
        acc = mulmod(acc, acc, m);
        if ((e >> bit) & 1)
            acc = mulmod(acc, b, m);
    }
    return acc;
}

u64 gcd64(u64 a, u64 b)
{
    while (b) {
        u64 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

u64 invmod(u64 a, u64 m)
{
    // Extended Euclid on signed 128-bit values.
    __int128 r0 = m, r1 = a % m, x0 = 0, x1 = 1;
    while (r1) {
        __int128 k = r0 / r1;
        __int128 t = r0 - k * r1;
        r0 = r1;
        r1 = t;
        t = x0 - k * x1;
        x0 = x1;
        x1 = t;
    }
    if (r0 != 1)
        return 0;
    if (x0 < 0)
        x0 += m;
    return (u64)x0;
}

u64 inv_mod_2_64(u64 n)
{
    // Newton iteration x <- x (2 - n x): each step doubles the correct bits;
    // x = n is correct to 3 bits for odd n.
    u64 x = n;
    for (int i = 0; i < 5; i++)
        x *= 2 - n * x;
    return x;
}

u32 inv_mod_2_32(u32 n)
{
    u32 x = n;
    for (int i = 0; i < 4; i++)
        x *= 2 - n * x;
    return x;
}

static bool strong_probable_prime(u64 n, u64 base)
{
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) {
        d >>= 1;
        r++;
    }
    u64 x = powmod(base, d, n);
    if (x == 1 || x == n - 1)
        return true;
    while (--r > 0) {
        x = mulmod(x, x, n);
        if (x == n - 1)
            return true;
    }
    return false;
}

bool is_prime(u64 x)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    static const u64 trial[] = {2,  3,  5,  7,  11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47,
                                53, 59, 61, 67, 71, 73, 79, 83, 89, 97, 101, 103, 107, 109, 113};
    if (x < 2)
        return false;
    for (u64 d : trial) {
        if (x == d)
            return true;
        if (x % d == 0)
            return false;
    }
    if (x < 113ULL * 113ULL)
        return true;
    const int nb = x < (1ULL << 32) ? 5 : 12;
    for (int i = 0; i < nb; i++)
        if (!strong_probable_prime(x, bases[i]))
            return false;
    return true;
}

u64 splitmix64_next(u64 &state)
{
    u64 z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int validate_pq(u64 p, u64 q, bool require_safe)
{
    const u64 lo = 1ULL << 31, hi = 1ULL << 32;
    if (p < lo || p >= hi || q < lo || q >= hi)
        return RSAPRNG_ERR_RANGE;
    if (p == q)
        return RSAPRNG_ERR_P_EQ_Q;
    if (!is_prime(p) || !is_prime(q))
        return RSAPRNG_ERR_NOT_PRIME;
    if (require_safe && (!is_prime((p - 1) / 2) || !is_prime((q - 1) / 2)))
        return RSAPRNG_ERR_NOT_PRIME;
    return RSAPRNG_OK;
}

static bool small_odd_exponent(u64 e) { return e >= 3 && (e & 1) && e < (1ULL << 32); }

int validate_pqe(u64 p, u64 q, u64 e, bool require_safe)
{
    const int rc = validate_pq(p, q, require_safe);
    if (rc)
        return rc;
    if (!small_odd_exponent(e) || gcd64(e, (p - 1) * (q - 1)) != 1)
        return RSAPRNG_ERR_E;
    return RSAPRNG_OK;
}

int validate_crt_exponents(u64 p, u64 q, u64 ep, u64 eq, bool require_safe)
{
    const int rc = validate_pq(p, q, require_safe);
    if (rc)
        return rc;
    if (!small_odd_exponent(ep) || !small_odd_exponent(eq) || gcd64(ep, p - 1) != 1 ||
        gcd64(eq, q - 1) != 1)
        return RSAPRNG_ERR_E;
    return RSAPRNG_OK;
}

void make_params(u64 p, u64 q, u64 e, u64 a, InstParams &o, u64 eq)
{
    if (eq == 0)
        eq = e;
    o = InstParams{};
    const u64 n = p * q;
    o.n = n;
    o.ninv = inv_mod_2_64(n);
    // The device exponentiates the plain residue with Montgomery products, so
    // the chain ends at m^e R^(1-e); one more product with R^e gives m^e.
    const u64 r64_mod_n = (u64)(((u128)1 << 64) % n);
    o.kn = powmod(r64_mod_n, e, n);
    o.r64 = r64_mod_n;
    o.p = (u32)p;
    o.q = (u32)q;
    o.pinv = inv_mod_2_32((u32)p);
    o.qinv = inv_mod_2_32((u32)q);
    // CRT route: the residue entering the chain is REDC(m) = m R^-1 (R = 2^32),
    // the chain ends at m^e R^(1-2e); the product with R^(2e) gives m^e.
    o.kp = (u32)powmod((1ULL << 32) % p, 2 * e, p);
    o.kq = (u32)powmod((1ULL << 32) % q, 2 * eq, q);
    o.garner = (u32)mulmod(invmod(q % p, p), (1ULL << 32) % p, p);
    o.e = (u32)e;
    o.eq = (u32)eq;
    o.a = (u32)a;
    o.root = (u32)root_index(a);
    // RN(n): n has 63 or 64 significant bits; round to 53 with ties to even.
    int bits = 64 - __builtin_clzll(n);
    int sh = bits - 53;
    u64 mn = n >> sh, rem = n & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
    if (rem > half || (rem == half && (mn & 1)))
        mn++;
    if (mn >> 53) {
        mn >>= 1;
        sh++;
    }
    o.en = sh;
    o.dn = (double)n;  // round to nearest even
    o.dnorm = mn << 11;
    // RN(1/RN(n)) from integers: 1/Mn has significand 2^105/Mn in (2^52, 2^53]
    // for Mn in [2^52, 2^53); round the exact quotient to nearest even.
    {
        const u128 num = (u128)1 << 105;
        u64 qq = (u64)(num / mn);
        const u64 rr = (u64)(num % mn);
        if (2 * (u128)rr > mn || (2 * (u128)rr == mn && (qq & 1)))
            qq++;
        // 1/RN(n) = (qq / 2^105) 2^-en; qq <= 2^53 (qq = 2^53 only when Mn = 2^52)
        o.recip = ldexp((double)qq, -105 - sh);
    }
    const u128 all = ~(u128)0;
    o.dv = (u64)(all / o.dnorm - ((u128)1 << 64));
    o.nsh = (u32)__builtin_clzll(n);
    o.vn = (u64)(all / (u128)(n << o.nsh) - ((u128)1 << 64));
}

int params_from_seed(u64 seed, int e_rule, u64 e_lo, u64 e_hi, u64 &p, u64 &q, u64 &e,
                     u64 &msg_seed)
{
    u64 st = seed;
    do {
        p = (splitmix64_next(st) >> 32) | 0x80000001ULL;
    } while (!is_prime(p));
    do {
        q = (splitmix64_next(st) >> 32) | 0x80000001ULL;
    } while (q == p || !is_prime(q));
    const u64 phi = (p - 1) * (q - 1);
    if (e_rule == RSAPRNG_E_SMALLEST || e_rule == RSAPRNG_E_AT_LEAST) {
        e = (e_rule == RSAPRNG_E_SMALLEST) ? 3 : (e_lo | 1);
        if (e < 3)
            e = 3;
        while (gcd64(e, phi) != 1)
            e += 2;
    } else if (e_rule == RSAPRNG_E_UNIFORM) {
        if (!(e_lo & 1) || e_hi < e_lo || e_lo < 3)
            return RSAPRNG_ERR_ARG;
        const u64 span = (e_hi - e_lo) / 2 + 1;
        // phi is even with at least one odd factor > 2 in general; an exponent
        // coprime to phi exists in any range containing a prime > phi's
        // factors, so the loop ends for the ranges in use.
        int guard = 0;
        do {
            e = e_lo + 2 * (splitmix64_next(st) % span);
            if (++guard > 1000000)
                return RSAPRNG_ERR_E;
        } while (gcd64(e, phi) != 1);
    } else {
        return RSAPRNG_ERR_ARG;
    }
    msg_seed = splitmix64_next(st);
    return RSAPRNG_OK;
}

}  // namespace rsaprng
