// Tagged words through which CTAs of one launch pass data without flags or fences: every
// 32-bit value travels in a 64-bit word whose upper half is a tag (the step the value
// belongs to). Words are written and read with relaxed GPU-scope 8-byte accesses, which are
// single-copy atomic, so a reader that finds the expected tag in a word also has that word's
// value. A reader that finds an older tag reads again, for a bounded clock budget.
#pragma once

#include <cstdint>

namespace pf {

__device__ __forceinline__ unsigned long long ll_word(unsigned int tag, float v) {
  return ((unsigned long long)tag << 32) | __float_as_uint(v);
}

// V (2 or 4) tagged words: V consecutive floats of one step, 16-byte aligned.
template <int V>
struct LLWords {
  unsigned long long w[V];
};

template <int V>
__device__ __forceinline__ void ll_store(unsigned long long* p, unsigned int tag, const float* v) {
  static_assert(V == 2 || V == 4, "two or four words");
#pragma unroll
  for (int k = 0; k < V; k += 2)
    asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p + k),
                 "l"(ll_word(tag, v[k])), "l"(ll_word(tag, v[k + 1]))
                 : "memory");
}

template <int V>
__device__ __forceinline__ LLWords<V> ll_load(const unsigned long long* p) {
  static_assert(V == 2 || V == 4, "two or four words");
  LLWords<V> q;
#pragma unroll
  for (int k = 0; k < V; k += 2)
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];"
                 : "=l"(q.w[k]), "=l"(q.w[k + 1])
                 : "l"(p + k)
                 : "memory");
  return q;
}

template <int V>
__device__ __forceinline__ bool ll_fresh(const LLWords<V>& q, unsigned int tag) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < V; ++k) ok = ok && (unsigned int)(q.w[k] >> 32) == tag;
  return ok;
}

template <int V>
__device__ __forceinline__ void ll_values(const LLWords<V>& q, float* v) {
#pragma unroll
  for (int k = 0; k < V; ++k) v[k] = __uint_as_float((unsigned int)q.w[k]);
}

// Read V tagged words until all carry `tag`; false once `budget` SM clocks have passed.
template <int V>
__device__ __forceinline__ bool ll_wait(const unsigned long long* p, unsigned int tag,
                                        long long budget, float* v) {
  const long long t0 = clock64();
  for (;;) {
    const LLWords<V> q = ll_load<V>(p);
    if (ll_fresh<V>(q, tag)) {
      ll_values<V>(q, v);
      return true;
    }
    if (clock64() - t0 > budget) return false;
  }
}

}  // namespace pf
