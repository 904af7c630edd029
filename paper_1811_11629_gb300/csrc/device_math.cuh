// Device arithmetic of the generator (arXiv:1811.11629 Sec. III-V), all exact.
//
//  - skip update a s mod Q (Eq. congruentialgenerator1) with Q = 2^63 - 25,
//    reduced by folding: 2^63 = 25 (mod Q), so hi 2^63 + lo = 25 hi + lo;
//  - message update (m + s) mod n with n in [2^62, 2^64) (Sec. IV);
//  - c = m^e mod n (Eq. encrypt2) either by CRT + Garner on two 32-bit
//    Montgomery exponentiations (Eq. CRTimplementation), or by one 64-bit
//    Montgomery exponentiation; both are exact, so both give the same c;
//  - r = RN(RN(c) / RN(n)) with the 1.0 guard (Eq. CodeFloatingPointStep),
//    either with IEEE double operations or with integers only.
#pragma once
#include <cstdint>

#include "host_params.hpp"

namespace rsaprng {
namespace dev {

constexpr u64 Q = 0x7FFFFFFFFFFFFFE7ULL;
constexpr u64 LOW63 = 0x7FFFFFFFFFFFFFFFULL;

// a s mod Q for a < 2^32 and s < Q: the product is below 2^95. With
// p0 = s_lo a and p1 = s_hi a + hi32(p0) (two widening multiply-adds, p1 <
// 2^64), a s = p1 2^32 + lo32(p0) = H 2^63 + L with H = p1 >> 31 < 2^33 and
// L = a s mod 2^63; 2^63 = 25 (mod Q) folds it to y = 25 H + L < 2^63 + 2^38,
// and y >= Q exactly when bit 63 of y + 25 is set, which then is y - Q.
__device__ __forceinline__ u64 mulmodQ_small(u64 s, u32 a)
{
    const u64 p0 = (u64)(u32)s * a;
    const u64 p1 = (u64)(u32)(s >> 32) * a + (p0 >> 32);
    const u64 H = p1 >> 31;
    const u64 L = ((p1 & 0x7FFFFFFFULL) << 32) | (u32)p0;
    const u64 y = H * 25 + L;
    const u64 z = y + 25;
    return (z >> 63) ? (z & LOW63) : y;
}

// acc += x with the carries out of 64 bits counted in cnt (the sum is
// acc + cnt 2^64).
__device__ __forceinline__ void add_carry_count(u64 &acc, u32 &cnt, u64 x)
{
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(acc), "+r"(cnt) : "l"(x));
}

// k r mod n for r < n by doubling and adding over the bits of k.
__device__ __forceinline__ u64 mulmod_small_count(u64 k, u64 r, u64 n)
{
    u64 t = 0;
    for (int b = k ? 63 - __clzll((long long)k) : -1; b >= 0; b--) {
        t = t + t >= n || t + t < t ? t + t - n : t + t;
        if ((k >> b) & 1) {
            const u64 u = t + r;
            t = (u < t || u >= n) ? u - n : u;
        }
    }
    return t;
}

// x y mod Q for x, y < Q (general 63-bit multiplier).
__device__ __forceinline__ u64 mulmodQ(u64 x, u64 y)
{
    const u64 lo = x * y;
    const u64 hi = __umul64hi(x, y);           // < 2^62
    const u64 H = (hi << 1) | (lo >> 63);      // < 2^63
    // 25 H + L63 in 128 bits
    const u64 t_lo = H * 25;
    const u64 t_hi = __umul64hi(H, 25ULL);
    const u64 y_lo = t_lo + (lo & LOW63);
    const u64 y_hi = t_hi + (y_lo < t_lo ? 1 : 0);  // y = y_hi 2^64 + y_lo < 26 2^63
    const u64 H2 = (y_hi << 1) | (y_lo >> 63);       // <= 25
    const u64 z = H2 * 25 + (y_lo & LOW63);           // < 2^63 + 2^10
    return z >= Q ? z - Q : z;
}

// (a + b) mod n for a, b < n < 2^64 (the sum may carry out of 64 bits).
__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 n)
{
    const u64 s = a + b;
    return (s < a || s >= n) ? s - n : s;
}

// a + b as a 64-bit representative of the sum's class mod n, not reduced:
// when the sum carries out of 64 bits, the dropped 2^64 is replaced by
// r64 = 2^64 mod n. With b < 2^63 the wrapped sum is below b, and r64 < 2^63
// (r64 = 2^64 - n for n > 2^63, else r64 < n < 2^63), so the second addition
// cannot carry. Messages are kept this way inside a tile: the exponentiation
// below needs only m mod p and m mod q, and n = 0 (mod p) and (mod q).
__device__ __forceinline__ u64 add_cong(u64 a, u64 b, u64 r64)
{
    const u64 t = a + b;
    return t < a ? t + r64 : t;
}

// x mod n for any 64-bit x: n >= 2^62, so x < 4n and three conditional
// subtractions suffice.
__device__ __forceinline__ u64 reduce_u64(u64 x, u64 n)
{
    x = x >= n ? x - n : x;
    x = x >= n ? x - n : x;
    return x >= n ? x - n : x;
}

// Montgomery reduction T 2^-32 mod p, p odd, pinv = p^-1 mod 2^32. With
// mq = T_lo pinv, mq p = T (mod 2^32) exactly, so T - mq p = (T_hi - hi(mq p))
// 2^32. hi(mq p) < p, so for any 64-bit T the result lies in [0, 2^32) and is
// congruent to T 2^-32; it is below p whenever T_hi < p (T < p 2^32), in
// particular for the product of any a < 2^32 with b < p.
__device__ __forceinline__ u32 redc32(u64 T, u32 p, u32 pinv)
{
    const u32 mq = (u32)T * pinv;
    const u32 u = __umulhi(mq, p);
    const u32 th = (u32)(T >> 32);
    const u32 r = th - u;
    return th < u ? r + p : r;
}
__device__ __forceinline__ u32 mont32(u32 a, u32 b, u32 p, u32 pinv)
{
    return redc32((u64)a * b, p, pinv);
}

// Montgomery product a b 2^-64 mod n, n odd, ninv = n^-1 mod 2^64. For any
// 64-bit a, b the result lies in [0, 2^64) and is congruent to a b 2^-64; it
// is below n whenever one factor is below n.
__device__ __forceinline__ u64 mont64(u64 a, u64 b, u64 n, u64 ninv)
{
    const u64 lo = a * b;
    const u64 hi = __umul64hi(a, b);
    const u64 mq = lo * ninv;
    const u64 u = __umul64hi(mq, n);
    const u64 r = hi - u;
    return hi < u ? r + n : r;
}

// c_j = m_j^e mod n for L messages by CRT (Eq. CRTimplementation): the
// residues enter as REDC(m) = m 2^-32 mod p (and mod q), left-to-right
// square-and-multiply runs on them with Montgomery products (Sec. I), the
// constants kp = 2^(64e) mod p, kq remove the Montgomery factors, and Garner's
// formula recombines: c = ((c_p - c_q) q^-1 mod p) q + c_q.
// m_j may be any 64-bit representative of the message's class mod n: the
// chain values stay below 2^32 and congruent, and the final product with
// kp < p (kq < q) returns the fully reduced residue.
// With CRT exponents (the q residue raised to eq != e, the paper's note on
// large exponents in Sec. V) both residues run in the same loop over the bits
// of the longer exponent: the residue whose exponent is shorter starts from
// the Montgomery form of 1 (2^32 mod p = 2^32 - p, below p as p > 2^31),
// which squaring leaves unchanged, so at its own top bit it becomes REDC(m)
// exactly as the ordinary chain starts; each residue multiplies on its own
// exponent's bits.
template <int L>
__device__ __forceinline__ void encrypt_crt(const u64 (&m)[L], u64 (&c)[L], const InstParams &P)
{
    const u32 p = P.p, q = P.q, pinv = P.pinv, qinv = P.qinv, e = P.e, eq = P.eq;
    const int top = 31 - __clz(e | eq);
    const bool p_on = (e >> top) & 1, q_on = (eq >> top) & 1;
    u32 yp[L], yq[L], zp[L], zq[L];
#pragma unroll
    for (int j = 0; j < L; j++) {
        yp[j] = redc32(m[j], p, pinv);
        yq[j] = redc32(m[j], q, qinv);
        zp[j] = p_on ? yp[j] : 0u - p;
        zq[j] = q_on ? yq[j] : 0u - q;
    }
    for (int bit = top - 1; bit >= 0; bit--) {
        u64 Tp[L], Tq[L];
#pragma unroll
        for (int j = 0; j < L; j++) {
            Tp[j] = (u64)zp[j] * zp[j];
            Tq[j] = (u64)zq[j] * zq[j];
        }
#pragma unroll
        for (int j = 0; j < L; j++) {
            zp[j] = redc32(Tp[j], p, pinv);
            zq[j] = redc32(Tq[j], q, qinv);
        }
        const bool mp = (e >> bit) & 1, mq = (eq >> bit) & 1;
        if (mp && mq) {
#pragma unroll
            for (int j = 0; j < L; j++) {
                Tp[j] = (u64)zp[j] * yp[j];
                Tq[j] = (u64)zq[j] * yq[j];
            }
#pragma unroll
            for (int j = 0; j < L; j++) {
                zp[j] = redc32(Tp[j], p, pinv);
                zq[j] = redc32(Tq[j], q, qinv);
            }
        } else if (mp) {
#pragma unroll
            for (int j = 0; j < L; j++)
                zp[j] = mont32(zp[j], yp[j], p, pinv);
        } else if (mq) {
#pragma unroll
            for (int j = 0; j < L; j++)
                zq[j] = mont32(zq[j], yq[j], q, qinv);
        }
    }
#pragma unroll
    for (int j = 0; j < L; j++) {
        const u32 cp = mont32(zp[j], P.kp, p, pinv);
        const u32 cq = mont32(zq[j], P.kq, q, qinv);
        const u32 cqp = cq >= p ? cq - p : cq;  // q < 2p
        u32 diff = cp - cqp;
        if (cp < cqp)
            diff += p;
        const u32 h = mont32(diff, P.garner, p, pinv);  // (c_p - c_q) q^-1 mod p
        c[j] = (u64)h * q + cq;
    }
}

// c_j = m_j^e mod n with 64-bit Montgomery products on the plain message:
// the chain ends at m^e 2^(64(1-e)); the product with kn = 2^(64e) mod n
// gives m^e mod n. As for the CRT route, m_j may be any 64-bit representative
// mod n; the final product with kn < n is fully reduced.
template <int L>
__device__ __forceinline__ void encrypt_mont64(const u64 (&m)[L], u64 (&c)[L], const InstParams &P)
{
    const u64 n = P.n, ninv = P.ninv;
    const u32 e = P.e;
    u64 z[L];
#pragma unroll
    for (int j = 0; j < L; j++)
        z[j] = m[j];
    const int top = 31 - __clz(e);
    for (int bit = top - 1; bit >= 0; bit--) {
#pragma unroll
        for (int j = 0; j < L; j++)
            z[j] = mont64(z[j], z[j], n, ninv);
        if ((e >> bit) & 1) {
#pragma unroll
            for (int j = 0; j < L; j++)
                z[j] = mont64(z[j], m[j], n, ninv);
        }
    }
#pragma unroll
    for (int j = 0; j < L; j++)
        c[j] = mont64(z[j], P.kn, n, ninv);
}

constexpr u64 ONE_MINUS_ULP_BITS = 0x3FEFFFFFFFFFFFFFULL;  // 1 - 2^-53

// The 1.0 guard for a non-negative double: the bit patterns of non-negative
// doubles are ordered as their values, so r >= 1.0 exactly when the pattern
// exceeds that of 1 - 2^-53. Tested on the integer pipe, not the FP64 one.
__device__ __forceinline__ double guard_below_one(double r)
{
    const u64 b = (u64)__double_as_longlong(r);
    return __longlong_as_double((long long)(b > ONE_MINUS_ULP_BITS ? ONE_MINUS_ULP_BITS : b));
}

// r = RN(RN(c)/RN(n)) with IEEE double conversion and division; dn = RN(n).
__device__ __forceinline__ double unit_fp64(u64 c, double dn)
{
    return guard_below_one(__ddiv_rn(__ull2double_rn(c), dn));
}

// The same value with the FP64 pipe but without a division: with the
// per-instance correctly rounded reciprocal y = RN(1/N) (N = RN(n)),
// q0 = RN(C y), the residual r = C - q0 N by one fused multiply-add, and the
// corrected quotient RN(q0 + r y) (Markstein's division by an FMA correction
// step, IBM J. Res. Dev. 34(1), 1990). Markstein's theorem needs q0 within
// one ulp of C/N; RN(C y) can be up to 1.5 ulps off when C's significand is
// below N's, but only where C/N is far from every midpoint between doubles,
// and there the correction step's error is still far smaller than that
// distance; near a midpoint q0 is always one of its two neighbours. So the
// result is RN(C/N) for every C, N (the library's tests check this
// exhaustively at reduced precision and on constructed near-midpoint
// quotients at full precision).
__device__ __forceinline__ double unit_recip(u64 c, double dn, double y)
{
    const double C = __ull2double_rn(c);
    const double q0 = __dmul_rn(C, y);
    const double r = __fma_rn(-q0, dn, C);
    return guard_below_one(__fma_rn(r, y, q0));
}

// 2/1 division by an invariant normalised divisor (Moller & Granlund,
// "Improved division by invariant integers", IEEE TC 2011, Algorithm 4):
// (u1 2^64 + u0) = q d + r for d >= 2^63, u1 < d and v = floor((2^128 - 1) /
// d) - 2^64.
__device__ __forceinline__ void div21(u64 u1, u64 u0, u64 d, u64 v, u64 &q, u64 &r)
{
    u64 q0 = v * u1;
    u64 q1 = __umul64hi(v, u1);
    q0 += u0;
    q1 += u1 + (q0 < u0 ? 1 : 0);
    q1 += 1;
    r = u0 - q1 * d;
    if (r > q0) {
        q1 -= 1;
        r += d;
    }
    if (r >= d) {
        q1 += 1;
        r -= d;
    }
    q = q1;
}

// The other reading of the division: r = RN(c / n) of the exact rational,
// with the same 1.0 guard. With N = n 2^s normalised (s = nsh) and C = c 2^s
// < N, the quotient digits of c/n in base 2^64 come from 2/1 divisions by N:
// (C, 0) / N = q1 rem r1, (r1, 0) / N = q2 rem r2, and c/n = (q1 2^64 + q2 +
// r2 / N) 2^-128. With lz leading zeros in q1 (q1 >= 1 since c/n > 2^-64),
// the significand is the 53 bits of (q1, q2) below bit 127 - lz; the bits
// under it and the remainder decide the rounding (ties to even). The second
// division is needed only when q1 alone holds fewer than 54 bits (lz > 10).
__device__ __forceinline__ double unit_exact(u64 c, const InstParams &P)
{
    if (c == 0)
        return 0.0;
    const u64 N = P.n << P.nsh, C = c << P.nsh;
    u64 q1, r1;
    div21(C, 0, N, P.vn, q1, r1);
    const int lz = __clzll(q1);
    u64 sig, rem, half;
    bool sticky;
    if (lz <= 10) {
        const int sh = 11 - lz;  // bits of q1 under the significand
        sig = q1 >> sh;
        rem = q1 & ((1ULL << sh) - 1);
        half = 1ULL << (sh - 1);
        sticky = r1 != 0;
    } else {
        u64 q2, r2;
        div21(r1, 0, N, P.vn, q2, r2);
        const int sh = 75 - lz;  // in [12, 64]: bits of q2 under the significand
        sig = (q1 << (64 - sh)) | (sh == 64 ? 0 : (q2 >> sh));
        rem = sh == 64 ? q2 : (q2 & ((1ULL << sh) - 1));
        half = 1ULL << (sh - 1);
        sticky = r2 != 0;
    }
    if (rem > half || (rem == half && (sticky || (sig & 1))))
        sig++;
    // value sig 2^(-53 - lz); sig in [2^52, 2^53], a rounded-up 2^53 carries
    // into the exponent field
    u64 bits = ((u64)(1021 - lz) << 52) + sig;
    if (bits > ONE_MINUS_ULP_BITS)
        bits = ONE_MINUS_ULP_BITS;
    return __longlong_as_double((long long)bits);
}

// The same value from integers only. RN(c) = Mc 2^Ec is rounded to 53 bits
// with ties to even; RN(n) = Mn 2^En is a per-instance constant. The
// significand quotient X / Mn with X = Mc 2^52 (Mc >= Mn) or Mc 2^53
// (Mc < Mn) lies in [2^52, 2^53); it is computed exactly, with remainder, by
// division by the invariant normalised divisor d = Mn 2^11 using the
// precomputed reciprocal v (Moller & Granlund, "Improved division by
// invariant integers", IEEE TC 2011, 2/1 division), then rounded to nearest
// even by comparing the remainder with d/2, and packed into a double.
__device__ __forceinline__ double unit_int(u64 c, const InstParams &P)
{
    if (c == 0)
        return 0.0;
    const int b = 64 - __clzll(c);
    u64 mc;
    int ec;
    if (b <= 53) {
        mc = c << (53 - b);
        ec = b - 53;
    } else {
        const int sh = b - 53;
        mc = c >> sh;
        const u64 rem = c & ((1ULL << sh) - 1);
        const u64 half = 1ULL << (sh - 1);
        if (rem > half || (rem == half && (mc & 1)))
            mc++;
        ec = sh;
        if (mc >> 53) {
            mc >>= 1;
            ec++;
        }
    }
    const u64 d = P.dnorm, v = P.dv;
    const u64 mn = d >> 11;
    u64 u1, u0;
    int E;
    if (mc >= mn) {
        u1 = mc >> 1;
        u0 = mc << 63;
        E = ec - P.en;
    } else {
        u1 = mc;
        u0 = 0;
        E = ec - P.en - 1;
    }
    u64 q1, r;
    div21(u1, u0, d, v, q1, r);
    const u64 halfd = d >> 1;
    if (r > halfd || (r == halfd && (q1 & 1)))
        q1++;
    if (q1 >> 53) {
        q1 >>= 1;
        E++;
    }
    u64 bits = ((u64)(E + 1023) << 52) | (q1 & ((1ULL << 52) - 1));
    if (bits > ONE_MINUS_ULP_BITS)
        bits = ONE_MINUS_ULP_BITS;
    return __longlong_as_double((long long)bits);
}

// The same value as unit_int, usually without the exact division. With X =
// Mc 2^11 and D = Mn 2^11 (both in [2^63, 2^64)) and v the invariant
// reciprocal of D, A = X + hi64(X v) approximates T = (X / D) 2^64 from
// below with an error T - A in [0, 3 + 2^-63): X + floor(X v / 2^64) lies in
// (T - 2 - 2^-63, T], and omitting the low 32x32 partial product of X v can
// lower it by one more. The 53-bit significand is A's top bits; the bits
// below it (g) decide the rounding. With an error below 4 units, g <= half - 4
// always rounds down and g > half always up; only g in [half - 3, half] is
// undecided, and there the exact routine decides. Rounding c
// to 53 bits uses the add-half-minus-one-plus-lsb rule (ties to even) on the
// left-normalised c; c < n < 2^64 - 2^35, so the addition cannot wrap.
__device__ __forceinline__ double unit_int_fast(u64 c, const InstParams &P)
{
    if (c == 0)
        return 0.0;
    const int lz = __clzll(c);
    const u64 t = c << lz;                                       // top bit set
    const u64 tr = t + (0x3FFULL + ((t >> 11) & 1));             // round at bit 11
    const bool carry = tr < t;                                   // rounded up to 2^64
    const u64 X = carry ? (1ULL << 63) : (tr & ~0x7FFULL);       // Mc << 11
    const int ec = 11 - lz + (carry ? 1 : 0);                    // RN(c) = (X >> 11) 2^ec
    const u64 v = P.dv;
    const u32 x0 = (u32)X, x1 = (u32)(X >> 32), v0 = (u32)v, v1 = (u32)(v >> 32);
    const u64 a = (u64)x1 * v0, b = (u64)x0 * v1;
    const u64 mid = a + b;
    const u64 hi = (u64)x1 * v1 + (mid >> 32) + ((u64)(mid < a) << 32);  // <= hi64(X v)
    const u64 A = X + hi;
    const bool ge1 = A < X;  // X/D >= 1 (bit 64 of X + hi)
    int E;
    u64 q, g, half;
    if (ge1) {  // significand = top 53 of the 65-bit A: bits 64..12
        q = (A >> 12) | (1ULL << 52);
        g = A & 0xFFF;
        half = 0x800;
        E = ec - P.en;
    } else {  // bits 63..11
        q = A >> 11;
        g = A & 0x7FF;
        half = 0x400;
        E = ec - P.en - 1;
    }
    if (g + 3 >= half && g <= half)
        return unit_int(c, P);  // the error could cross the halfway point
    q += (g > half) ? 1 : 0;
    // q in [2^52, 2^53]; adding q to the exponent field one below carries a
    // rounded-up 2^53 into the exponent.
    u64 bits = ((u64)(E + 1022) << 52) + q;
    if (bits > ONE_MINUS_ULP_BITS)
        bits = ONE_MINUS_ULP_BITS;
    return __longlong_as_double((long long)bits);
}

}  // namespace dev
}  // namespace rsaprng
