// Vector moves of a thread's V consecutive values of one plane (float4 / float2 / double2 accesses),
// for kernels whose register lanes hold consecutive nodes. The caller checks VecIo::ok first; where
// it fails (a wrapped or clamped node, an unaligned place or plane) the kernel moves node by node.
#pragma once

#include <cuda_runtime.h>
#include <string.h>

namespace lbm {

template <int BYTES>
struct VecWord;
template <>
struct VecWord<16> {
  using type = float4;
};
template <>
struct VecWord<8> {
  using type = float2;
};

template <typename R, int V>
struct VecIo {
  static constexpr int kBytes = V * (int)sizeof(R);
  // Whole 16-byte accesses, or one 8-byte access for two floats; one value moves as it is.
  static constexpr bool kOn = V > 1 && (kBytes % 16 == 0 || kBytes == 8);
  static constexpr int kChunk = kBytes % 16 == 0 ? 16 : 8;
  static constexpr int kElems = kChunk / (int)sizeof(R);

  // Values pos0 ... pos0 + V - 1 of every plane of length N (planes N apart) lie inside the plane
  // and start on a kChunk-byte boundary.
  __device__ static bool ok(const R* base, long long pos0, long long N) {
    return kOn && pos0 >= 0 && pos0 + V <= N && (pos0 % kElems) == 0 && (N % kElems) == 0 &&
           (reinterpret_cast<unsigned long long>(base) % kChunk) == 0;
  }
  __device__ static void load(const R* p, R (&t)[V]) {
    using W = typename VecWord<kChunk>::type;
#pragma unroll
    for (int c = 0; c < kBytes / kChunk; ++c) {
      const W w = reinterpret_cast<const W*>(p)[c];
      memcpy(&t[c * kElems], &w, kChunk);
    }
  }
  __device__ static void store(R* p, const R (&t)[V]) {
    using W = typename VecWord<kChunk>::type;
#pragma unroll
    for (int c = 0; c < kBytes / kChunk; ++c) {
      W w;
      memcpy(&w, &t[c * kElems], kChunk);
      reinterpret_cast<W*>(p)[c] = w;
    }
  }
};

}  // namespace lbm
