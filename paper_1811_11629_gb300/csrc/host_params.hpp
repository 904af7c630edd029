// Host-side number theory and per-instance constants for the generator
// (arXiv:1811.11629 Sec. III-V). Plain C++ with unsigned __int128.
#pragma once
#include <cstdint>

namespace rsaprng {

using u64 = uint64_t;
using u32 = uint32_t;
using u128 = unsigned __int128;

constexpr u64 kQ = 0x7FFFFFFFFFFFFFE7ULL;  // 2^63 - 25 (Sec. V)

// Allowed skip multipliers (restricted primitive roots mod Q). Index 0 is the
// default. The table index is stored per instance to select power tables.
constexpr int kNumRoots = 14;
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

// Device-side record of one instance's fixed parameters (112 bytes). Field
// meaning is documented at the kernels that read it.
struct alignas(16) InstParams {
    u64 n;       // p q
    u64 ninv;    // n^{-1} mod 2^64 (Montgomery, R = 2^64)
    u64 kn;      // 2^(64 e) mod n: undoes the Montgomery factor of the chain
    u64 dv;      // floor((2^128 - 1) / dnorm) - 2^64 (invariant division)
    u64 dnorm;   // significand of RN(n) shifted to bit 63: Mn << 11
    u32 p, q;
    u32 pinv, qinv;  // p^{-1}, q^{-1} mod 2^32
    u32 kp, kq;      // 2^(64 e) mod p, mod q
    u32 garner;      // (q^{-1} mod p) * 2^32 mod p
    u32 e;
    u32 a;           // skip multiplier
    u32 root;        // index into kRoots (power tables)
    int32_t en;      // RN(n) = Mn * 2^en, Mn in [2^52, 2^53)
    u32 pad;
    double dn;       // RN(n) as a double
    double recip;    // RN(1 / RN(n)), the correctly rounded reciprocal
    u64 r64;         // 2^64 mod n
};
static_assert(sizeof(InstParams) == 112, "InstParams layout");

// Validation codes mirror RSAPRNG_ERR_*.
int validate_pqe(u64 p, u64 q, u64 e, bool require_safe);
// Fills the constants; p, q, e already validated; a allowed.
void make_params(u64 p, u64 q, u64 e, u64 a, InstParams &out);

// The seeded parameter rule (documented in rsaprng.h).
int params_from_seed(u64 seed, int e_rule, u64 e_lo, u64 e_hi, u64 &p, u64 &q, u64 &e,
                     u64 &msg_seed);

// a^k mod Q.
inline u64 powQ(u64 a, u64 k) { return powmod(a, k, kQ); }

}  // namespace rsaprng
