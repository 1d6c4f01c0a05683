// Internal declarations of the radix-sort kernels of libvrs (sm_103a).
#pragma once

#include "vrs_internal.cuh"

namespace vrs {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys
constexpr int kSortWarps = kSortThreads / 32;

struct SortArgs {
    const unsigned long long *keys_in;
    const uint32_t *vals_in;
    unsigned long long *keys_out;
    uint32_t *vals_out;
    uint32_t *counts;     // [kRadix][G]
    uint32_t *totals;     // [kRadix]
    const DevStatus *st;
    unsigned long long cap;
    int shift;
    int G;
    uint32_t digit_mask;  // 255, or fewer bits on a last pass that ends inside a byte
};

struct DownSmem {
    unsigned long long keys[kSortTile];
    uint32_t vals[kSortTile];
    uint32_t whist[kSortWarps][kRadix + 1];
    uint32_t dstart[kRadix];
    uint32_t gbase[kRadix];
    uint32_t tcnt[kRadix];
    uint32_t wtot[kSortWarps];
};

__global__ void __launch_bounds__(kSortThreads) k_upsweep(const SortArgs a);
__global__ void __launch_bounds__(1024) k_scan_digits(const SortArgs a);
__global__ void __launch_bounds__(kSortThreads) k_downsweep(const SortArgs a);

}  // namespace vrs
