// span.cuh -- the rank space the merge levels run over.
//
// One hull: the n ranks of one sorted cloud.  Many hulls at once: every cloud
// sorted into its own block of 2^L_c ranks (L_c = ceil(log2 n_c)), the blocks
// laid out largest first so that each starts at a multiple of its size.  A
// node of level l <= L_c then lies inside its cloud's block, so the bottom-up
// merge steps of Sec. 2 (nodes of aligned power-of-two blocks, the "kernel
// index math" of Sec. 3) run over all clouds at once: one launch per level
// merges every cloud's nodes of that level, each independent of the others.
#pragma once
#include <stdint.h>

namespace hull3d {

constexpr int SPAN_SHIFT = 13;  // clouds of the multi-cloud rank space hold more than 4096 points

struct Span {
    int64_t n;            // ranks in use: one cloud's n, or the end of the last block
    const int32_t *blk;   // nullptr: one cloud.  Else the cloud owning each 2^SPAN_SHIFT ranks (-1: none)
    const int64_t *cbase; // per cloud: first rank of its block
    const int64_t *cend;  // per cloud: one past its last rank (block start + n_c)
    const int32_t *ctop;  // per cloud: its root level L_c
    const int32_t *cstat; // per cloud: nonzero once an input error was found (its nodes are skipped)
};

// The node of `level` whose first rank is lo (a multiple of 2^level): false
// when there is none there (past the ranks in use, in a cloud's padding,
// above its cloud's root, or in a failed cloud); else hi = the node's end,
// min(lo + 2^level, end), with end the end of its cloud.
__host__ __device__ __forceinline__ bool node_span(const Span &sp, int level, int64_t lo, int64_t &hi, int64_t &end)
{
    if (lo >= sp.n) return false;
    end = sp.n;
    if (sp.blk) {
        const int32_t c = sp.blk[lo >> SPAN_SHIFT];
        if (c < 0 || sp.ctop[c] < level || sp.cstat[c]) return false;
        end = sp.cend[c];
        if (lo >= end) return false;
    }
    hi = lo + (1ll << level) < end ? lo + (1ll << level) : end;
    return true;
}

__host__ __device__ __forceinline__ bool node_span(const Span &sp, int level, int64_t lo, int64_t &hi)
{
    int64_t end;
    return node_span(sp, level, lo, hi, end);
}

// One cloud of n ranks.
inline Span single_span(int64_t n) { return Span{ n, nullptr, nullptr, nullptr, nullptr, nullptr }; }

}  // namespace hull3d
