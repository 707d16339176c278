// lbve_sched.cuh -- the quasi-logarithmic history grid of Sec. III in closed form.
//
// B blocks (b = 1 coarsest .. B finest; index bb = b - 1) of C points; points of block b are
// 2^(B-b) steps apart and the gap from the oldest point of block b+1 to the newest of block b is
// 2^(B-b) as well.  Every block starts full of rest points.  Block B receives the new point every
// step; block b < B receives the merged point of block b+1 every 2^(B-b) steps.  A full receiving
// block b > 1 first hands its two oldest points on, merged (older point's E, averaged kappa); a full
// block 1 drops its oldest point.  Counting receipts gives the whole state in closed form, identical
// at every node, so the device computes it from the step index t alone (no host schedule, nothing to
// upload, and a captured CUDA graph stays valid for any t).
//
// Storage: each block is a ring of C slots; its newest point sits at ring slot `head`, the k-th newest
// at (head - k) mod C.  Points never move inside the ring; a merge copies one point into the coarser
// block's ring (done by the history kernel after its sweep).
#pragma once
#include <stdint.h>

#define LBVE_MAXB 16

#if defined(__CUDACC__)
#define LBVE_HD __host__ __device__ __forceinline__
#else
#define LBVE_HD inline
#endif

struct BlockStep {
    int head_prev, count_prev;  // ring slot of the newest point and number of points after step t-1
    int head_new, count_new;    // the same after step t
    int recv;                   // block receives a point at step t
    int evict;                  // ... and is full: b > 1 merges its two oldest, b = 1 drops its oldest
    int spacing;                // 2^(B-b)
    int age_prev;               // age (at t-1) of the block's newest point
};

// Ring head and count of block bb after step t (t = -1: the initial, full state).
LBVE_HD void sched_block_state(int B, int C, long long t, int bb, int* head, int* count) {
    if (t < 0) {
        *head = C - 1;
        *count = C;
        return;
    }
    const long long r = t >> (B - 1 - bb);   // index of the latest receipt
    // (the 32-bit remainder for any receipt index below 2^32, the same value as the 64-bit one)
    *head = r <= 0xFFFFFFFFll ? (int)((unsigned)r % (unsigned)C) : (int)(r % C);
    *count = (bb == 0) ? C : ((r & 1) == 0 ? C - 1 : C);
}

// State of block bb in step t >= 0, every field but age_prev.
LBVE_HD void sched_block(int B, int C, long long t, int bb, BlockStep* sb) {
    const int sp = 1 << (B - 1 - bb);
    int hp, cp, hn, cn;
    sched_block_state(B, C, t - 1, bb, &hp, &cp);
    sched_block_state(B, C, t, bb, &hn, &cn);
    const int recv = (t & (long long)(sp - 1)) == 0;
    sb->head_prev = hp;
    sb->count_prev = cp;
    sb->head_new = hn;
    sb->count_new = cn;
    sb->recv = recv;
    sb->evict = recv && cp == C;
    sb->spacing = sp;
}

// Per-block state transition of step t >= 0.  The age of block bb's newest point, finest block first: the
// ages spanned by every finer block (its points times its spacing, less one) plus the gaps between blocks.
LBVE_HD void sched_step(int B, int C, long long t, BlockStep* s) {
    int age = 0;
    for (int bb = B - 1; bb >= 0; --bb) {
        sched_block(B, C, t, bb, &s[bb]);
        if (bb != B - 1) age += s[bb].spacing;                // gap to the oldest point of the finer block
        s[bb].age_prev = age;
        age += (s[bb].count_prev - 1) * s[bb].spacing;        // age of the block's oldest point
    }
}

#if defined(__CUDACC__)
// sched_step computed by a CTA: lane bb < B of warp 0 fills block bb, and the ages follow as warp suffix sums,
// age_prev(bb) = sum over b > bb of (count_prev(b) - 1) spacing(b) + sum over bb <= b < B - 1 of spacing(b).
// CTAs of fewer than 32 threads let thread 0 run sched_step.  Every thread of the CTA calls it; the states
// are valid after the caller's next __syncthreads().
__device__ __forceinline__ void sched_step_cta(int B, int C, long long t, BlockStep* s) {
    if (blockDim.x < 32) {
        if (threadIdx.x == 0) sched_step(B, C, t, s);
        return;
    }
    if (threadIdx.x >= 32) return;
    const int bb = threadIdx.x;
    int term = 0, gap = 0;
    if (bb < B) {
        BlockStep b;
        sched_block(B, C, t, bb, &b);
        term = (b.count_prev - 1) * b.spacing;
        gap = bb < B - 1 ? b.spacing : 0;
        s[bb] = b;
    }
    int st = term, sg = gap;   // inclusive suffix sums over lanes bb .. 31
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a1 = __shfl_down_sync(0xffffffffu, st, o);
        const int a2 = __shfl_down_sync(0xffffffffu, sg, o);
        if (bb + o < 32) {
            st += a1;
            sg += a2;
        }
    }
    if (bb < B) s[bb].age_prev = st - term + sg;
}
#endif

// Role of ring slot j of block bb during step t, for a point already in memory (the point created at
// step t is not in memory yet).  Returns the trapezoidal weight (0 = slot takes no part: empty, or
// the newer half of a merge, or dropped), its age at step t, and `partner` = slot index (bb*C + j')
// whose kappa is averaged into this one (the older half of a merge), else -1.
LBVE_HD float sched_slot_role(const BlockStep* s, int C, int bb, int j, int* age, int* partner) {
    const BlockStep& b = s[bb];
    int k = b.head_prev - j;
    if (k < 0) k += C;
    *partner = -1;
    *age = 0;
    if (k >= b.count_prev) return 0.0f;
    *age = b.age_prev + k * b.spacing + 1;
    if (b.evict) {
        if (k == C - 1) {
            if (bb == 0) return 0.0f;                          // dropped from the coarsest block
            int j2 = b.head_prev - (C - 2);
            if (j2 < 0) j2 += C;
            *partner = bb * C + j2;
            return (float)(2 * b.spacing);                     // newest point of block bb-1
        }
        if (k == C - 2 && bb > 0) return 0.0f;                 // newer half of the merge
    }
    const int kn = k + b.recv;
    if (kn == b.count_new - 1)                                 // the block's oldest point
        return bb > 0 ? 1.5f * (float)b.spacing : 0.5f * (float)b.spacing;
    return (float)b.spacing;
}
