// Distance keys of the packed solver state, shared by the GOVM kernels.
#pragma once

#include <cstdint>

#include "dawn_common.cuh"

namespace dawn {

// Distance keys, monotone in the distance so that the packed atomicMin
// orders by distance: uint32 distances are their own key; non-negative
// float32 distances are keyed by their bit pattern; signed int32 distances
// by their offset-binary code (sign bit flipped).  `zero` is the key of a
// source, `inf` of an unreachable vertex; `out` turns a key back into the
// bits of the output distance.
template <int WT>
struct Key;
template <>
struct Key<DAWN_W_U32> {
  static constexpr uint32_t inf = kInfKeyU32;
  static constexpr uint32_t zero = 0u;
  static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) { return d + w; }
  static __device__ __forceinline__ uint32_t out(uint32_t k) { return k; }
};
template <>
struct Key<DAWN_W_F32> {
  static constexpr uint32_t inf = kInfKeyF32;
  static constexpr uint32_t zero = 0u;
  static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
    return __float_as_uint(__fadd_rn(__uint_as_float(d), __uint_as_float(w)));
  }
  static __device__ __forceinline__ uint32_t out(uint32_t k) { return k; }
};
template <>
struct Key<DAWN_W_I32> {
  static constexpr uint32_t inf = 0xFFFFFFFFu;   // INT32_MAX: unreachable
  static constexpr uint32_t zero = 0x80000000u;  // distance 0
  static __device__ __forceinline__ uint32_t add(uint32_t d, uint32_t w) {
    return (uint32_t)((int32_t)(d ^ 0x80000000u) + (int32_t)w) ^ 0x80000000u;
  }
  static __device__ __forceinline__ uint32_t out(uint32_t k) { return k ^ 0x80000000u; }
};

}  // namespace dawn
