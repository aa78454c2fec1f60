// prg.cuh -- the counter PRG every dealt value and MAC-check coefficient
// comes from.
//
// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) in counter form: output i of a generator whose
// state starts at `key` is mix(key + (i + 1) * GAMMA), with the published
// mixing function (xor-shift 30, multiply, xor-shift 27, multiply,
// xor-shift 31).  Streams: key(seed, stream) = sm64(seed, stream), with
// stream = kind << 56 | role << 48 | party << 40 | sub (sub < 2^40).
// Field elements: p61 takes the top 61 bits of sm64(key, j); p127 takes
// sm64(key, 2j) as the low word and the top 63 bits of sm64(key, 2j+1) as the
// high word; the value p itself maps to 0.  p = 2^32-5 takes the top 32 bits
// of sm64(key, j), minus p when they are p or above.
#pragma once
#include <cstdint>
#include "field.cuh"

namespace spdz {

constexpr uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t sm64(uint64_t key, uint64_t i) {
    return sm_mix(key + (i + 1) * SM_GAMMA);
}

enum Role : uint64_t { ROLE_SECRET = 0, ROLE_VAL_SHARE = 1, ROLE_MAC_SHARE = 2 };

__host__ __device__ __forceinline__ uint64_t stream_id(uint64_t kind, uint64_t role,
                                                       uint64_t party, uint64_t sub) {
    return (kind << 56) | (role << 48) | (party << 40) | (sub & ((1ull << 40) - 1));
}

__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm64(seed, stream);
}

template <class F> struct Draw;

template <> struct Draw<F61> {
    __device__ __forceinline__ static F61::T at(uint64_t key, uint64_t j) {
        return F61::from_draw(sm64(key, j));
    }
};

template <> struct Draw<F32> {
    __device__ __forceinline__ static F32::T at(uint64_t key, uint64_t j) {
        return F32::from_draw(sm64(key, j));
    }
};

template <> struct Draw<F127> {
    __device__ __forceinline__ static F127::T at(uint64_t key, uint64_t j) {
        return F127::from_draws(sm64(key, 2 * j), sm64(key, 2 * j + 1));
    }
};

}  // namespace spdz
