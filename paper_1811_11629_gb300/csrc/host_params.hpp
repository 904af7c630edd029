// Host-side number theory and per-instance constants for the generator
// (arXiv:1811.11629 Sec. III-V). Plain C++ with unsigned __int128.
#pragma once
#include <cstdint>

namespace rsaprng {

using u64 = uint64_t;
using u32 = uint32_t;
using u128 = unsigned __int128;

constexpr u64 kQ = 0x7FFFFFFFFFFFFFE7ULL;  // 2^63 - 25 (Sec. V)

// Allowed skip multipliers (restricted primitive roots mod Q, and 1 for the
// unit / constant skip). Index 0 is the default. The table index is stored
// per instance to select power tables.
constexpr int kNumRoots = 15;
extern const u64 kRoots[kNumRoots];
int root_index(u64 a);  // -1 if not allowed

u64 mulmod(u64 a, u64 b, u64 m);
u64 powmod(u64 b, u64 e, u64 m);
u64 gcd64(u64 a, u64 b);
u64 invmod(u64 a, u64 m);  // 0 if not invertible
u64 inv_mod_2_64(u64 n);   // n odd: n^{-1} mod 2^64
u32 inv_mod_2_32(u32 n);   // n odd: n^{-1} mod 2^32
bool is_prime(u64 x);      // Sec. V: trial division + deterministic Rabin-Miller

// SplitMix64 step (Steele, Lea & Flood 2014).
u64 splitmix64_next(u64 &state);

// Device-side record of one instance's fixed parameters (128 bytes). Field
// meaning is documented at the kernels that read it.
struct alignas(16) InstParams {
    u64 n;       // p q
    u64 ninv;    // n^{-1} mod 2^64 (Montgomery, R = 2^64)
    u64 kn;      // 2^(64 e) mod n: undoes the Montgomery factor of the chain
    u64 dv;      // floor((2^128 - 1) / dnorm) - 2^64 (invariant division)
    u64 dnorm;   // significand of RN(n) shifted to bit 63: Mn << 11
    u32 p, q;
    u32 pinv, qinv;  // p^{-1}, q^{-1} mod 2^32
    u32 kp, kq;      // 2^(64 e) mod p, 2^(64 eq) mod q
    u32 garner;      // (q^{-1} mod p) * 2^32 mod p
    u32 e;           // exponent (of the p residue when eq differs)
    u32 a;           // skip multiplier
    u32 root;        // index into kRoots (power tables)
    int32_t en;      // RN(n) = Mn * 2^en, Mn in [2^52, 2^53)
    u32 eq;          // exponent of the q residue (= e unless CRT exponents)
    double dn;       // RN(n) as a double
    double recip;    // RN(1 / RN(n)), the correctly rounded reciprocal
    u64 r64;         // 2^64 mod n
    u64 vn;          // floor((2^128 - 1) / (n << nsh)) - 2^64 (exact division by n)
    u32 nsh;         // leading zeros of n
    u32 pad;
};
static_assert(sizeof(InstParams) == 128, "InstParams layout");

// Validation codes mirror RSAPRNG_ERR_*.
int validate_pq(u64 p, u64 q, bool require_safe);
int validate_pqe(u64 p, u64 q, u64 e, bool require_safe);
// CRT exponents: p, q as validate_pq; e_p, e_q odd in [3, 2^32) with
// gcd(e_p, p - 1) = gcd(e_q, q - 1) = 1.
int validate_crt_exponents(u64 p, u64 q, u64 ep, u64 eq, bool require_safe);
// Fills the constants; p, q, e (and eq) already validated; a allowed. eq = 0
// means eq = e.
void make_params(u64 p, u64 q, u64 e, u64 a, InstParams &out, u64 eq = 0);

// The seeded parameter rule (documented in rsaprng.h).
int params_from_seed(u64 seed, int e_rule, u64 e_lo, u64 e_hi, u64 &p, u64 &q, u64 &e,
                     u64 &msg_seed);

// a^k mod Q.
inline u64 powQ(u64 a, u64 k) { return powmod(a, k, kQ); }

}  // namespace rsaprng
