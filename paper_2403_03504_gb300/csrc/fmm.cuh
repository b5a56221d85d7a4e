// Fast Multipole Method for the ForceAtlas2 repulsion (Section 3.2.1).
#pragma once
#include "bgl_internal.cuh"

namespace bgl {

struct FmmPlan;

// Buffers for the FMM of component c (sized for its node count); reused
// across iterations.
FmmPlan *fmm_create(bgl_graph *g, const bgl_params *p, int64_t c);
void fmm_destroy(FmmPlan *pl);

// f[q - fbase] <- kr m_q sum_j m_j (p_q - p_j) / |p_q - p_j|^2 (+ fa[q - fbase]
// when fa is not null) for every position q of the component, with
// xy[q - qbase] the positions.  The kernel that adds fa first waits for the
// event fa_ready (if not null) on the calling stream.  Launches only (no
// host synchronisation), so it can be captured in a CUDA graph.
void fmm_repulsion(FmmPlan *pl, const float2 *xy, int64_t qbase, float2 *f, int64_t fbase, const float2 *fa = nullptr,
                   cudaEvent_t fa_ready = nullptr);

// Fused ForceAtlas2 iteration for a run whose only component is this plan's
// (Section 3.2): the combine pass also sums swing and traction and its last
// block sets s_G (and the statistics), and fmm_update_root moves the points
// and makes the next evaluation's root square in the same pass, so the
// evaluations skip their bounding-box kernel.  Arrays are indexed q - fbase
// (positions q - qbase) as in fmm_repulsion.
struct FmmFuse {
    const float2 *fprev = nullptr;   // F_{t-1}, indexed like f
    int variant = 0;
    double tau = 1.0;
    double *sg = nullptr;            // s_G of the component
    double *stats = nullptr;         // optional: swing, traction, s_G per iteration
    int *iter = nullptr;             // iteration counter of the statistics
    float ks = 0.1f, ksmax = 10.f;
    int *bad = nullptr;              // set when a position becomes non-finite
};
void fmm_fuse(FmmPlan *pl, const FmmFuse &fz);
// the root square of positions xy (before the first fused evaluation)
void fmm_root(FmmPlan *pl, const float2 *xy, int64_t qbase);
// p += s F, F_{t-1} <- F for every point, and the next root square
void fmm_update_root(FmmPlan *pl, float2 *xy, int64_t qbase, const float2 *f, float2 *fprev, int64_t fbase);

// Counts and per-phase device times of `reps` evaluations (synchronises);
// out[15]: boxes, leaves, depth, P2P pairs, M2L translations, M2P terms,
// P2L terms, then milliseconds of: points (bbox, keys, sort, gather), tree,
// lists, upward pass, downward pass, near field, far field (one stream),
// and of a whole evaluation in the concurrent schedule.
void fmm_profile(FmmPlan *pl, const float2 *xy, int64_t qbase, int reps, double *out);

// Radix passes the plan's next sort skips (0 or 2): chosen on the device from
// the depth of the previous evaluation's tree, so it is part of the state a
// resumed run needs (reading and setting synchronise the stream).
int fmm_sortskip(FmmPlan *pl);
void fmm_set_sortskip(FmmPlan *pl, int skip);

// Error bits raised on the device since the plan was made (synchronises):
// 1 a bounded wait gave up, 2 list capacity exceeded, 4 box capacity
// exceeded, 8 non-finite bounding box.
int fmm_error(FmmPlan *pl);

}  // namespace bgl
