// vec.cuh -- 16-byte vector access to party-major share rows: four p = 2^32-5
// elements, two p61 elements or one p127 element per access (the caller
// checks that the rows are 16-byte aligned).  STREAM loads use the
// evict-first hint for data read once.
#pragma once
#include <type_traits>

#include "field.cuh"

namespace spdz {

template <class F, int V, bool STREAM>
__device__ __forceinline__ void vld(const typename F::T *p, typename F::T (&out)[V]) {
    if constexpr (std::is_same_v<F, F32>) {
        static_assert(V == 1 || V == 4, "p32 moves one or four elements per access");
        if constexpr (V == 4) {
            const uint4 *q = reinterpret_cast<const uint4 *>(p);
            const uint4 t = STREAM ? __ldcs(q) : *q;
            out[0] = t.x; out[1] = t.y; out[2] = t.z; out[3] = t.w;
        } else {
            out[0] = STREAM ? __ldcs(reinterpret_cast<const unsigned int *>(p)) : *p;
        }
    } else if constexpr (F::WORDS == 1) {
        if constexpr (V == 2) {
            const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(p);
            ulonglong2 t = STREAM ? __ldcs(q) : *q;
            out[0] = t.x;
            out[1] = t.y;
        } else {
            const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
            out[0] = STREAM ? __ldcs(q) : *q;
        }
    } else {
        static_assert(V == 1, "p127 moves one element per access");
        const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(p);
        ulonglong2 t = STREAM ? __ldcs(q) : *q;
        out[0] = {t.x, t.y};
    }
}

template <class F, int V>
__device__ __forceinline__ void vst(typename F::T *p, const typename F::T (&in)[V]) {
    if constexpr (std::is_same_v<F, F32>) {
        if constexpr (V == 4)
            *reinterpret_cast<uint4 *>(p) = make_uint4(in[0], in[1], in[2], in[3]);
        else
            *p = in[0];
    } else if constexpr (F::WORDS == 1) {
        if constexpr (V == 2) {
            *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(in[0], in[1]);
        } else {
            *reinterpret_cast<unsigned long long *>(p) = in[0];
        }
    } else {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(in[0].lo, in[0].hi);
    }
}

}  // namespace spdz
