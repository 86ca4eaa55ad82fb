// Descriptor sources for kernels that run one product or a whole batch.
//
// A kernel body takes the descriptor of one unit of work (a product, a
// sub-product set, a normalization job...) and a block index local to it.
// The same body runs
//   * for one product: One<Args> holds the descriptor by value (kernel
//     parameter space), the grid is that product's blocks;
//   * for a batch: Many<Args> points at descriptors in device memory and at
//     the prefix sums of their block counts; a CTA finds its descriptor by
//     binary search.
#pragma once

#include <stdint.h>

namespace ks {

template <class T>
struct One {
  T d;
  __device__ __forceinline__ const T &locate(int64_t bid, int64_t &local) const {
    local = bid;
    return d;
  }
  // also the index of the descriptor (always 0)
  __device__ __forceinline__ const T &locate(int64_t bid, int64_t &local, int &idx) const {
    local = bid;
    idx = 0;
    return d;
  }
  // the descriptor of a known index (no search)
  __device__ __forceinline__ const T &at(int, int64_t bid, int64_t &local) const {
    local = bid;
    return d;
  }
};

template <class T>
struct Many {
  const T *d;
  const int64_t *prefix;  // n + 1 entries, prefix[0] = 0
  int n;
  __device__ __forceinline__ const T &locate(int64_t bid, int64_t &local) const {
    int lo = 0, hi = n - 1;
    while (lo < hi) {  // last q with prefix[q] <= bid
      const int mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= bid)
        lo = mid;
      else
        hi = mid - 1;
    }
    local = bid - prefix[lo];
    return d[lo];
  }
  __device__ __forceinline__ const T &locate(int64_t bid, int64_t &local, int &idx) const {
    const T &r = locate(bid, local);
    idx = (int)(&r - d);
    return r;
  }
  // the descriptor of a known index (no search)
  __device__ __forceinline__ const T &at(int idx, int64_t bid, int64_t &local) const {
    local = bid - prefix[idx];
    return d[idx];
  }
};

}  // namespace ks
