// All-pairs BatMap comparison (the hot loop of Sec. III-B): tile shapes,
// schedule construction and launch.
#pragma once

#include "common.cuh"

namespace bm {

// Tile shapes of the compare kernel.  A CTA of 256 threads owns a tile of
// TR rows x TC columns (each thread 8 rows x MC columns).  Staged shapes
// (stages > 0) stream the column width in stages of KC words through shared
// memory; direct shapes (stages == 0) stream 4-word steps into registers.
struct ShapeDesc {
    uint32_t id;   // 1-based; 0 = automatic
    uint32_t TR, TC, MC, KC, stages;  // (MC: columns per thread)
    double eff;    // relative throughput per padded word-pair (scheduler prior)
};

constexpr int NUM_SHAPES = 16;
extern const ShapeDesc SHAPES[NUM_SHAPES];

// Number of SMs of the current device (cached).
int device_sms();

// Build the compare work units of one set (fills S->units, longest first,
// and uploads them).  `shape_eff` (NULL = built-in prior) gives the relative
// throughput of each shape (autotuner); `force_shape` (1..NUM_SHAPES) pins
// one shape; target_cost <= 0 picks about 8 units per SM.
void build_schedule(batmap_set *S);
void schedule_units(const batmap_set *S, uint32_t force_shape, const double *shape_eff,
                    double target_cost, std::vector<WorkUnit> *out);

// Estimated cost of a unit (padded word-pairs / shape efficiency) and the
// order used by every launch: units of the main shapes first, then those of
// the one-column shapes 14..16 (small_shape), each part longest first.
double unit_cost(const WorkUnit &u);
void sort_units(std::vector<WorkUnit> *units);
bool small_shape(uint32_t shape);
uint32_t main_units(const std::vector<WorkUnit> &units);  // length of the first part

// Launch the persistent compare kernels over `count` units at d_units (any
// mix of instances) ordered by sort_units, the first nmain of the main
// shapes: one kernel per part, pulling work from d_counters[0] and
// d_counters[1] (zeroed by the caller).  One CTA per SM.  d_stamps (optional,
// set by the caller to {~0, 0}) receives the earliest CTA start and latest CTA
// end in globaltimer nanoseconds (timing inside captured graphs).
void launch_compare(const InstView *d_views, const WorkUnit *d_units, uint32_t count, uint32_t nmain,
                    uint32_t *d_counters, cudaStream_t st, unsigned long long *d_stamps = nullptr);

// Sets the kernel's shared-memory attribute (call before stream capture).
void prepare_compare();

// Shared-memory bytes of one shape (for occupancy and launch).
size_t compare_smem_bytes(uint32_t shape_idx);

}  // namespace bm
