// Karras hierarchy of sorted Morton keys (Karras 2012, Sec. 4): the
// per-node construction shared by the LBVH build (build.cu) and the SAH
// builds' fallback below their depth cap (sah.cu).  Internal header.
#pragma once

#include "rg_internal.cuh"

namespace rg {
namespace {

template <class K>
__device__ __forceinline__ int clz_key(K x);
template <>
__device__ __forceinline__ int clz_key<uint32_t>(uint32_t x) { return __clz(x); }
template <>
__device__ __forceinline__ int clz_key<uint64_t>(uint64_t x) { return __clzll(x); }

// augmented common-prefix length (Karras 2012, Sec. 4); -1 outside [0, n).
// KS: the sorted keys, any type indexable by position (a pointer, or a view
// through an index array).
template <class KS>
__device__ __forceinline__ int delta(const KS& k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const auto a = k[i], b = k[j];
    using K = decltype(a + 0u);
    if (a != b) return clz_key<K>((K)(a ^ b));
    return (int)(8 * sizeof(K)) + __clz((uint32_t)i ^ (uint32_t)j);
}

// Internal node i of the Karras hierarchy over n sorted keys: its children
// (bit 31 marks a leaf) into child_base[i * stride], its key range into
// ranges (optional), its children's parent entries (optional).  For a
// segment of a larger tree (node_off > 0), node and leaf indices are offset by
// node_off and leaf_off, parents are laid out for n_all leaves, and the
// segment root's own parent entry is left alone.
template <class KS>
__device__ __forceinline__ void karras_node(const KS& keys, uint32_t n, int64_t i,
                                            uint32_t* __restrict__ child_base, int stride, uint32_t* __restrict__ parents,
                                            uint32_t* __restrict__ ranges, uint32_t node_off = 0, uint32_t leaf_off = 0,
                                            uint32_t n_all = 0) {
    if (n_all == 0) n_all = n;
    const int64_t N = n;
    int d = (delta(keys, N, i, i + 1) - delta(keys, N, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(keys, N, i, i - d);
    int64_t lmax = 2;
    while (delta(keys, N, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(keys, N, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(keys, N, i, j);
    int64_t s = 0, t;
    int64_t div = 2;
    do {
        t = (l + div - 1) / div;
        if (delta(keys, N, i, i + (s + t) * d) > dnode) s += t;
        div <<= 1;
    } while (t > 1);
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    uint32_t left = (lo == gamma) ? (kLeaf | (leaf_off + (uint32_t)gamma)) : node_off + (uint32_t)gamma;
    uint32_t right = (hi == gamma + 1) ? (kLeaf | (leaf_off + (uint32_t)(gamma + 1))) : node_off + (uint32_t)(gamma + 1);
    const size_t me = node_off + (size_t)i;
    child_base[me * stride] = left;
    child_base[me * stride + 1] = right;
    if (ranges) {
        ranges[2 * me] = leaf_off + (uint32_t)lo;
        ranges[2 * me + 1] = leaf_off + (uint32_t)hi;
    }
    if (parents) {
        parents[(left & kLeaf) ? (size_t)(n_all - 1) + (left & ~kLeaf) : left] = (uint32_t)me;
        parents[(right & kLeaf) ? (size_t)(n_all - 1) + (right & ~kLeaf) : right] = (uint32_t)me;
        if (i == 0 && node_off == 0) parents[0] = kNone;
    }
}

}  // namespace
}  // namespace rg
