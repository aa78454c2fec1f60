// field.cuh -- exact arithmetic modulo the Mersenne primes 2^61-1 and 2^127-1,
// and modulo 2^32-5 (the prime of the paper's evaluation, Sec. IV-A).
//
// Every function takes canonical operands in [0, p) and returns a canonical
// result.  Mersenne products are reduced with the identity 2^k == 1 (mod
// 2^k - 1): the double-width product is split at bit k and the halves are
// added, followed by one conditional subtract.  Products mod 2^32-5 use
// 2^32 == 5 twice.  Device products use 64-bit mul.lo / mul.hi (lowered to
// 32-bit IMAD sequences by the compiler).
#pragma once
#include <cstdint>

namespace spdz {

// ------------------------------------------------------------------ p61
struct F61 {
    using T = uint64_t;
    static constexpr int WORDS = 1;
    static constexpr uint64_t P = (1ull << 61) - 1;

    __host__ __device__ __forceinline__ static T zero() { return 0; }
    __host__ __device__ __forceinline__ static bool is_zero(T a) { return a == 0; }
    __host__ __device__ __forceinline__ static T add(T a, T b) {
        T s = a + b;                 // < 2^62
        return s >= P ? s - P : s;
    }
    __host__ __device__ __forceinline__ static T sub(T a, T b) {
        T d = a - b;
        return a >= b ? d : d + P;
    }
    __host__ __device__ __forceinline__ static T neg(T a) { return a == 0 ? 0 : P - a; }
    // (hi:lo) < 2^122  ->  (hi:lo) mod p
    __device__ __forceinline__ static T reduce122(uint64_t lo, uint64_t hi) {
        // x = (x >> 61) * 2^61 + (x & p), and 2^61 == 1: both halves are <= p
        // for x <= (p-1)^2, and their sum is < 2p.
        T s = (lo & P) + ((hi << 3) | (lo >> 61));
        return s >= P ? s - P : s;
    }
    __device__ __forceinline__ static T mul(T a, T b) {
        return reduce122(a * b, __umul64hi(a, b));
    }
    // Field element from a 64-bit PRG word: the top 61 bits, p maps to 0.
    __host__ __device__ __forceinline__ static T from_draw(uint64_t d) {
        T v = d >> 3;
        return v == P ? 0 : v;
    }
    __device__ __forceinline__ static T ld(const T *p) { return *p; }
    __device__ __forceinline__ static void st(T *p, T v) { *p = v; }
};

// ------------------------------------------------------------- 2^32 - 5
// Elements are uint32 words.  (hi:lo) = hi * 2^32 + lo == 5 hi + lo.
struct F32 {
    using T = uint32_t;
    static constexpr int WORDS = 1;
    static constexpr uint32_t P = 4294967291u;   // 2^32 - 5

    __host__ __device__ __forceinline__ static T zero() { return 0; }
    __host__ __device__ __forceinline__ static bool is_zero(T a) { return a == 0; }
    __host__ __device__ __forceinline__ static T add(T a, T b) {
        const uint64_t s = (uint64_t)a + b;     // < 2p
        return (T)(s >= P ? s - P : s);
    }
    __host__ __device__ __forceinline__ static T sub(T a, T b) {
        return a >= b ? a - b : (T)((uint64_t)a + P - b);
    }
    __host__ __device__ __forceinline__ static T neg(T a) { return a == 0 ? 0 : P - a; }
    // x < 2^64 -> x mod p: x == 5 * (x >> 32) + (x & (2^32 - 1)) < 2^35,
    // once more (< 2^32 + 35), then one conditional subtract
    __host__ __device__ __forceinline__ static T reduce64(uint64_t x) {
        x = 5ull * (x >> 32) + (x & 0xffffffffull);
        x = 5ull * (x >> 32) + (x & 0xffffffffull);
        return (T)(x >= P ? x - P : x);
    }
    __host__ __device__ __forceinline__ static T mul(T a, T b) { return reduce64((uint64_t)a * b); }
    // Field element from a 64-bit PRG word: the top 32 bits, minus p when
    // they are p or above.
    __host__ __device__ __forceinline__ static T from_draw(uint64_t d) {
        const uint32_t v = (uint32_t)(d >> 32);
        return v >= P ? v - P : v;
    }
    __device__ __forceinline__ static T ld(const T *p) { return *p; }
    __device__ __forceinline__ static void st(T *p, T v) { *p = v; }
};

// Deferred reduction for p61: a sum of a few 122-bit products (and canonical
// terms) is kept as an exact 128-bit integer and reduced once.
struct W61 {
    uint64_t lo = 0, hi = 0;
    // += a * b, a and b below 2^61
    __device__ __forceinline__ void mac(uint64_t a, uint64_t b) {
        const uint64_t pl = a * b, ph = __umul64hi(a, b);
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(pl), "l"(ph));
    }
    __device__ __forceinline__ void add(uint64_t a) {
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(a));
    }
    // the sum mod 2^61 - 1, for a sum below 2^124: two folds with 2^61 == 1
    // (the first leaves less than 2^61 + 2^63, the second at most p + 4),
    // then one conditional subtract
    __device__ __forceinline__ uint64_t reduce() const {
        uint64_t s = (lo & F61::P) + ((hi << 3) | (lo >> 61));
        s = (s & F61::P) + (s >> 61);
        return s >= F61::P ? s - F61::P : s;
    }
};

// An exact sum of many p61 products, reduced once: three 64-bit words hold
// up to 2^64 products of operands below 2^64.  With 2^61 == 1 (mod p),
// w1 2^64 == 8 w1 and w2 2^128 == 64 w2, each split at bit 61.
struct S61 {
    uint64_t w0 = 0, w1 = 0, w2 = 0;
    __device__ __forceinline__ void add(uint64_t a) {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
            : "+l"(w0), "+l"(w1), "+l"(w2) : "l"(a));
    }
    __device__ __forceinline__ void mac(uint64_t a, uint64_t b) {
        const uint64_t pl = a * b, ph = __umul64hi(a, b);
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, 0;"
            : "+l"(w0), "+l"(w1), "+l"(w2) : "l"(pl), "l"(ph));
    }
    __device__ __forceinline__ uint64_t reduce() const {
        // six pieces, each below 2^61: the sum is below 2^64
        uint64_t s = (w0 & F61::P) + (w0 >> 61) + ((w1 << 3) & F61::P) + (w1 >> 58) + ((w2 << 6) & F61::P) +
                     (w2 >> 55);
        s = (s & F61::P) + (s >> 61);
        return s >= F61::P ? s - F61::P : s;
    }
};

// c + a1 b1 + a2 b2 (+ a3 b3) mod p with one reduction where the field allows
// it: p61 sums the 122-bit products exactly in 128 bits (below 2^124);
// p = 2^32-5 folds each 64-bit product to 5 hi + lo (below 2^35) and sums in
// 64 bits; p127 reduces each product (an exact 256-bit sum measured no
// faster: its cost is the 128 x 128-bit products themselves).
template <class F> struct Fma {
    __device__ __forceinline__ static typename F::T f2(typename F::T c, typename F::T a1, typename F::T b1,
                                                       typename F::T a2, typename F::T b2) {
        return F::add(c, F::add(F::mul(a1, b1), F::mul(a2, b2)));
    }
    __device__ __forceinline__ static typename F::T f3(typename F::T c, typename F::T a1, typename F::T b1,
                                                       typename F::T a2, typename F::T b2, typename F::T a3,
                                                       typename F::T b3) {
        return F::add(f2(c, a1, b1, a2, b2), F::mul(a3, b3));
    }
};
template <> struct Fma<F61> {
    __device__ __forceinline__ static uint64_t f2(uint64_t c, uint64_t a1, uint64_t b1, uint64_t a2, uint64_t b2) {
        W61 w;
        w.add(c);
        w.mac(a1, b1);
        w.mac(a2, b2);
        return w.reduce();
    }
    __device__ __forceinline__ static uint64_t f3(uint64_t c, uint64_t a1, uint64_t b1, uint64_t a2, uint64_t b2,
                                                  uint64_t a3, uint64_t b3) {
        W61 w;
        w.add(c);
        w.mac(a1, b1);
        w.mac(a2, b2);
        w.mac(a3, b3);
        return w.reduce();
    }
};
template <> struct Fma<F32> {
    __device__ __forceinline__ static uint64_t fold(uint64_t x) { return 5ull * (x >> 32) + (x & 0xffffffffull); }
    __device__ __forceinline__ static uint32_t f2(uint32_t c, uint32_t a1, uint32_t b1, uint32_t a2, uint32_t b2) {
        return F32::reduce64((uint64_t)c + fold((uint64_t)a1 * b1) + fold((uint64_t)a2 * b2));
    }
    __device__ __forceinline__ static uint32_t f3(uint32_t c, uint32_t a1, uint32_t b1, uint32_t a2, uint32_t b2,
                                                  uint32_t a3, uint32_t b3) {
        return F32::reduce64((uint64_t)c + fold((uint64_t)a1 * b1) + fold((uint64_t)a2 * b2) + fold((uint64_t)a3 * b3));
    }
};

// ----------------------------------------------------------------- p127
struct u128v {
    uint64_t lo, hi;
};

struct F127 {
    using T = u128v;
    static constexpr int WORDS = 2;
    static constexpr uint64_t PLO = ~0ull;
    static constexpr uint64_t PHI = (1ull << 63) - 1;

    __host__ __device__ __forceinline__ static T zero() { return {0, 0}; }
    __host__ __device__ __forceinline__ static bool is_zero(T a) { return (a.lo | a.hi) == 0; }
    __host__ __device__ __forceinline__ static bool is_p(T a) { return a.lo == PLO && a.hi == PHI; }

    // s < 2^128 -> s mod p, by one fold of bit 127 and one compare with p.
    __host__ __device__ __forceinline__ static T fold128(uint64_t lo, uint64_t hi) {
        uint64_t top = hi >> 63;
        hi &= PHI;
        uint64_t nlo = lo + top;
        hi += (nlo < lo);
        lo = nlo;
        // now (hi:lo) <= p
        if (lo == PLO && hi == PHI) return {0, 0};
        return {lo, hi};
    }
    __host__ __device__ __forceinline__ static T add(T a, T b) {
        uint64_t lo = a.lo + b.lo;
        uint64_t hi = a.hi + b.hi + (lo < a.lo);   // < 2^128
        return fold128(lo, hi);
    }
    __host__ __device__ __forceinline__ static T sub(T a, T b) {
        uint64_t lo = a.lo - b.lo;
        uint64_t borrow = a.lo < b.lo;
        uint64_t hi = a.hi - b.hi - borrow;
        bool neg = (a.hi < b.hi) || (a.hi == b.hi && borrow);
        if (neg) {                                  // add p (mod 2^128)
            uint64_t nlo = lo + PLO;
            hi = hi + PHI + (nlo < lo);
            lo = nlo;
        }
        return {lo, hi};
    }
    __host__ __device__ __forceinline__ static T neg(T a) { return sub(zero(), a); }

    // 256-bit product of a, b < 2^127 reduced mod p: x = H*2^127 + L,
    // 2^127 == 1, so x == H + L with H, L < 2^127.
    __device__ __forceinline__ static T mul(T a, T b) {
        uint64_t p00l = a.lo * b.lo, p00h = __umul64hi(a.lo, b.lo);
        uint64_t p01l = a.lo * b.hi, p01h = __umul64hi(a.lo, b.hi);
        uint64_t p10l = a.hi * b.lo, p10h = __umul64hi(a.hi, b.lo);
        uint64_t p11l = a.hi * b.hi, p11h = __umul64hi(a.hi, b.hi);
        uint64_t w0 = p00l, w1, w2, w3;
        asm("add.cc.u64  %0, %3, %4;\n\t"
            "addc.cc.u64 %1, %5, %6;\n\t"
            "addc.u64    %2, %7, 0;\n\t"
            : "=l"(w1), "=l"(w2), "=l"(w3)
            : "l"(p00h), "l"(p01l), "l"(p01h), "l"(p11l), "l"(p11h));
        asm("add.cc.u64  %0, %0, %3;\n\t"
            "addc.cc.u64 %1, %1, %4;\n\t"
            "addc.u64    %2, %2, 0;\n\t"
            : "+l"(w1), "+l"(w2), "+l"(w3)
            : "l"(p10l), "l"(p10h));
        // L = bits 0..126, H = bits 127..253
        uint64_t Llo = w0, Lhi = w1 & PHI;
        uint64_t Hlo = (w1 >> 63) | (w2 << 1);
        uint64_t Hhi = (w2 >> 63) | (w3 << 1);
        uint64_t lo = Llo + Hlo;
        uint64_t hi = Lhi + Hhi + (lo < Llo);       // < 2^128
        return fold128(lo, hi);
    }
    // Field element from two PRG words: low word, then the top 63 bits of the
    // second word as the high word; p maps to 0.
    __host__ __device__ __forceinline__ static T from_draws(uint64_t d0, uint64_t d1) {
        T v{d0, d1 >> 1};
        return is_p(v) ? zero() : v;
    }
    __device__ __forceinline__ static T ld(const T *p) {
        ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
        return {v.x, v.y};
    }
    __device__ __forceinline__ static void st(T *p, T v) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(v.lo, v.hi);
    }
};

// Deferred reduction for p127: an exact sum below 2^190 in three words,
// reduced once.  A product of a, b < 2^127 enters as three word-aligned
// pieces congruent to it: with a = a1 2^64 + a0, b = b1 2^64 + b0 and
// m = a1 b0 + a0 b1 = mh 2^64 + ml (below 2^128), 2^128 == 2 (mod p) gives
//   a b == a0 b0 + ml 2^64 + 2 (a1 b1 + mh),
// each piece below 2^128, so no product is folded at bit 127 on its own.
struct W127 {
    uint64_t w0 = 0, w1 = 0, w2 = 0;
    // += c, c below 2^128
    __device__ __forceinline__ void add(u128v c) {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, 0;"
            : "+l"(w0), "+l"(w1), "+l"(w2) : "l"(c.lo), "l"(c.hi));
    }
    // += another three-word sum
    __device__ __forceinline__ void add(const W127 &q) {
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
            : "+l"(w0), "+l"(w1), "+l"(w2) : "l"(q.w0), "l"(q.w1), "l"(q.w2));
    }
    // A three-word value congruent to a * b (mod p), a and b below 2^127
    // (below 3 * 2^128): the product's pieces are summed here, so several
    // products can be formed independently before they meet in one sum.
    __device__ __forceinline__ static W127 prod(u128v a, u128v b) {
        const uint64_t p0l = a.lo * b.lo, p0h = __umul64hi(a.lo, b.lo);
        uint64_t ml = a.hi * b.lo, mh = __umul64hi(a.hi, b.lo);
        const uint64_t ql = a.lo * b.hi, qh = __umul64hi(a.lo, b.hi);
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(ml), "+l"(mh) : "l"(ql), "l"(qh));
        uint64_t tl = a.hi * b.hi, th = __umul64hi(a.hi, b.hi);     // a1 b1 < 2^126
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(tl), "+l"(th) : "l"(mh));   // < 2^127
        W127 q;
        q.w0 = tl << 1;
        q.w1 = (th << 1) | (tl >> 63);
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, 0, 0;\n\t"
            "add.cc.u64 %1, %1, %5;\n\taddc.u64 %2, %2, 0;"
            : "+l"(q.w0), "+l"(q.w1), "=l"(q.w2) : "l"(p0l), "l"(p0h), "l"(ml));
        return q;
    }
    // += a * b (mod p), a and b below 2^127
    __device__ __forceinline__ void mac(u128v a, u128v b) { add(prod(a, b)); }
    // The sum mod 2^127 - 1: w2 2^128 == 2 w2; the 128-bit rest and its carry
    // are folded at bit 127 (below 2^127 + 3 after the fold), and s >= p
    // exactly when s + 1 reaches 2^127, where s - p = s + 1 - 2^127.
    __device__ __forceinline__ u128v reduce() const {
        uint64_t x0 = w0, x1 = w1, c;
        asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, 0, 0;"
            : "+l"(x0), "+l"(x1), "=l"(c) : "l"(w2 << 1));
        uint64_t s0 = x0, s1 = x1 & F127::PHI;
        asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(s0), "+l"(s1) : "l"((x1 >> 63) + 2 * c));
        uint64_t t0 = s0, t1 = s1;
        asm("add.cc.u64 %0, %0, 1;\n\taddc.u64 %1, %1, 0;" : "+l"(t0), "+l"(t1));
        if (t1 >> 63) return {t0, t1 & F127::PHI};
        return {s0, s1};
    }
};

template <> struct Fma<F127> {
    __device__ __forceinline__ static u128v f2(u128v c, u128v a1, u128v b1, u128v a2, u128v b2) {
        W127 w = W127::prod(a1, b1);
        w.add(W127::prod(a2, b2));
        w.add(c);
        return w.reduce();
    }
    __device__ __forceinline__ static u128v f3(u128v c, u128v a1, u128v b1, u128v a2, u128v b2, u128v a3, u128v b3) {
        W127 w = W127::prod(a1, b1), v = W127::prod(a2, b2);
        w.add(W127::prod(a3, b3));
        v.add(c);
        w.add(v);
        return w.reduce();
    }
};

}  // namespace spdz
