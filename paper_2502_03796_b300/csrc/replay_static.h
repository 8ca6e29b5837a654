// replay_static.h - the static-baseline kernel (replay_static.cu): work items, launch
// parameters and host entry points.
#pragma once
#include <vector>

#include "magus_internal.h"

namespace magus {

// One CTA of the static kernel: blocks [first, first + count) of 2048 deltas of a trace
// charged in `parts` CTAs.
struct StaticItem {
    uint32_t trace, first, count, parts;
};
struct StaticParams {
    const uint32_t *traces;
    const uint64_t *offsets;
    const uint64_t *lengths;
    int32_t n_traces;
    int32_t n_pols;            // pair index = trace * n_pols + policy
    const DevPolicy *pols;
    const int32_t *lit;        // device: policy indices; the pinned ones are replayed here
    int32_t n_lit;
    int32_t n_items;           // CTAs, one per item
    const StaticItem *items;
    unsigned long long *acc;   // [n_traces][2][MAGUS_MAX_LEVELS + 1]: counts, sums per r (zeroed)
    uint32_t *arrived;         // [n_traces] parts finished (zeroed)
    DevModel model;
    double *energy, *edp, *time;
    uint64_t *n_changes, *change_hash, *n_hf;
};
// Parts of 2048-delta blocks for the static kernel: about four waves of CTAs, longest first.
void static_items(const std::vector<uint64_t> &lengths, int sms, int K, std::vector<StaticItem> *out);
cudaError_t launch_replay_static(const StaticParams &p, cudaStream_t stream);

}  // namespace magus
