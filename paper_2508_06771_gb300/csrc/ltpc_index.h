// ltpc_index.h -- index arithmetic of the cluster cell kernel, shared by the
// device code and the host-side self-check (no CUDA types in here).
//
// A cell of n particles is processed by a cluster of C CTAs.  Three
// distributions of work over the C CTAs are used:
//   * home slices   : perm positions [H(r), H(r+1)), H(r) = floor(r n / C);
//                     the CTA loads these particles' ids and velocities
//                     (coalesced) and writes them back at the end.
//   * bucket ranges : sort buckets [B(r), B(r+1)), B(r) = floor(r nb / C),
//                     nb = n (one bucket per particle on average); the CTA
//                     keeps those bucket counters.
//   * pair slots    : slots [Q(r), Q(r+1)), Q(r) = floor(r half / C),
//                     half = ceil(n / 2); slot p covers pairing-order
//                     positions 2p and 2p+1, so the CTA owns positions
//                     [2 Q(r), min(2 Q(r+1), n)) and no pair straddles CTAs.
// For a range split R(r) = floor(r T / C) of T items, the owner of item t is
// the largest r with R(r) <= t, which is floor(((t + 1) C - 1) / T); it
// satisfies R(owner) <= t < R(owner + 1) even when some ranges are empty.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define LTPC_HD __host__ __device__ __forceinline__
#else
#define LTPC_HD static inline
#endif

namespace ltpc {

LTPC_HD uint32_t split_begin(uint32_t r, uint32_t total, uint32_t C)
{
    return (uint32_t)(((uint64_t)r * total) / C);
}

LTPC_HD uint32_t split_owner(uint32_t t, uint32_t total, uint32_t C)
{
    return (uint32_t)((((uint64_t)t + 1u) * C - 1u) / total);
}

LTPC_HD uint32_t n_buckets(uint32_t n) { return n < 1 ? 1u : n; }
LTPC_HD uint32_t n_half(uint32_t n) { return (n + 1u) / 2u; }

// First pairing-order position owned by CTA r.
LTPC_HD uint32_t pos_begin(uint32_t r, uint32_t n, uint32_t C)
{
    return 2u * split_begin(r, n_half(n), C);
}

LTPC_HD uint32_t pos_end(uint32_t r, uint32_t n, uint32_t C)
{
    uint32_t e = 2u * split_begin(r + 1u, n_half(n), C);
    return e < n ? e : n;
}

LTPC_HD uint32_t pos_owner(uint32_t q, uint32_t n, uint32_t C)
{
    return split_owner(q >> 1, n_half(n), C);
}

// Largest cell a cluster of C CTAs with `capl` positions per CTA can hold.
LTPC_HD uint32_t cluster_capacity(uint32_t C, uint32_t capl) { return C * capl; }

}  // namespace ltpc
